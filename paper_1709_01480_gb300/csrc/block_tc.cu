// Block-diagonal body operators on the tensor cores (Sec. 3.4, Eqs.
// preconditionerGMRES, approximate-body-mobility, M-block-inverse; Eqs.
// Gprecond-decomp, Gprecond-precompute for the Lanczos blocks).
//
// Every body b carries the same reference block B_ref (2 n_p x 2 n_p: M_ref^+ for
// the preconditioner, G_ref or G_ref^+ for the near-field square root), so the
// block-diagonal operator is one contraction G = B_ref Z over all bodies, with
// Z[:, b] = R_b^T in_b the body's vector rotated into its frame.  One kernel does
// the rotation, the contraction and the per-body epilogue:
//
//   TC_ROTATE     out_b = R_b g_b                        (Lanczos G, G^+ blocks)
//   TC_BODYFRAME  g_b as FP32, unrotated                 (input of the coarse level)
//   TC_PRECOND    the body solve of the preconditioner: U' = -N~ (R^T r_U + K_ref^T g),
//                 mu = R (g + H U'), U = R U'  (H = M_ref^+ K_ref, N~ = (K^T M^+ K)^-1)
//
// Tensor-core form.  tcgen05.mma kind::tf32, M = 128 rows of B_ref per tile (one or
// two tiles), N = 16 bodies per CTA, K = 8 per instruction, FP32 accumulators in
// tensor memory.  FP32 accuracy from TF32 operands by the three-term split
// a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi (a_hi = a rounded to TF32, a_lo = a - a_hi):
// the dropped a_lo b_lo and the TF32 truncation of the low parts are ~2^-22 relative.
// B_ref's two parts are laid out once, at setup, in the operand layout below and
// streamed through shared memory in chunks of 32 K-columns by bulk copies (double-
// buffered, mbarrier completion); the CTA's Z tile (16 bodies x all K) is formed in
// shared memory by the CTA's threads.
//
// Operand layout (K-major, no swizzle): core matrices of 8 rows x 16 bytes (4 FP32)
// stored as 128 contiguous bytes; the next core matrix along K at +128 bytes
// (leading byte offset), the next along M/N at +SBO (stride byte offset).
//
// Every wait is bounded (0.25 s on the global timer): on expiry the kernel records
// the failure in *err, waits (bounded) for its own copies, frees its tensor memory
// and returns without writing results; the host reports FBIM_ERR_TIMEOUT.
#include <cstdint>
#include <cstring>
#include <vector>

#include "fbim_internal.h"
#include "solver.cuh"

namespace fbim {

namespace {

constexpr int TC_N = 16;           // bodies per CTA (MMA N)
constexpr int TC_KC = 32;          // K columns per streamed chunk
constexpr int TC_TILE_FLOATS = 128 * TC_KC;  // one M-tile x one chunk x one part
constexpr unsigned long long TC_WAIT_NS = 250000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Shared-memory matrix descriptor: start address, leading (K) and stride (M/N) byte
// offsets, fixed field 0b001 at bits 46-48, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Bounded wait for the phase with the given parity; false (and *err set, err non-null)
// on expiry.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int* err) {
    const uint64_t t0 = globaltimer();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
        if (globaltimer() - t0 > TC_WAIT_NS) {
            if (err) atomicOr(err, 1);
            return false;
        }
    }
}

__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ float tf32_hi(float x) {
    uint32_t u;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
    return __uint_as_float(u & 0xFFFFE000u);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, int acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 16 consecutive accumulator columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[TC_N]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

struct TcArgs {
    const float* A;       // B_ref in the chunked operand layout [KC][2][MT][128 x 32]
    int n_b, n_p, n2, KP, MT, KC;
    const double* rot;    // [n_b][2] (cos, sin)
    const double* in;     // [n_b * n_p][2] (then [n_b][3] r_U for TC_PRECOND)
    const double* ref;    // [n_p][2] reference nodes (TC_PRECOND)
    const float* H;       // [3][n2] M_ref^+ K_ref (TC_PRECOND)
    double nt[9];         // N~_ref row-major (TC_PRECOND)
    double* out;          // [n_b * n_p][2] (TC_ROTATE: out; TC_PRECOND: mu)
    double* out_U;        // [n_b][3] (TC_PRECOND)
    float* out_g;         // [n_b][n2] (TC_BODYFRAME)
    int* err;             // failure flag
};

enum { TC_ROTATE = 0, TC_BODYFRAME = 1, TC_PRECOND = 2 };

template <int MODE>
__global__ void __launch_bounds__(128, 1) k_block_tc(TcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int KP = a.KP, MT = a.MT, KC = a.KC, n2 = a.n2, n_p = a.n_p;
    // carve: B tile (2 parts x 16 x KP floats), A stages (2 x 2 parts x MT tiles), barriers
    float* sB = reinterpret_cast<float*>(smem_raw);
    const int b_part = TC_N * KP;  // floats per part
    float* sA = sB + 2 * b_part;
    const int stage_floats = 2 * MT * TC_TILE_FLOATS;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sA + 2 * stage_floats);  // full[2], empty[2], done
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 5);
    float* red = reinterpret_cast<float*>(tmem_slot + 4);                  // [4 MT][48]
    double* Us = reinterpret_cast<double*>(red + 4 * 2 * 48);              // [16][3]
    const int b0 = blockIdx.x * TC_N;
    // an earlier launch failed: leave the outputs alone (one decision for the whole CTA)
    if (__syncthreads_or(tid == 0 ? *a.err : 0)) return;

    if (tid == 0) {
        for (int i = 0; i < 5; ++i) mbar_init(&bars[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(smem_u32(tmem_slot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    __syncthreads();
    const unsigned chunk_bytes = (unsigned)(stage_floats * sizeof(float));
    if (tid == 0) {  // the first two chunks of B_ref in flight while the Z tile forms
        for (int c = 0; c < 2 && c < KC; ++c) {
            mbar_expect_tx(&bars[c], chunk_bytes);
            bulk_copy(sA + c * stage_floats, a.A + (size_t)c * stage_floats, chunk_bytes, &bars[c]);
        }
    }
    // Z tile: z = R_b^T in_b for the CTA's bodies, split into TF32 high and low parts;
    // element (n, k) at (n/8) 8 KP + (k/4) 32 + (n%8) 4 + k%4 of each part
    for (int i = tid; i < TC_N * (KP / 2); i += blockDim.x) {
        const int n = i / (KP / 2), j = i - n * (KP / 2);  // node j: K indices 2j, 2j+1
        const int b = b0 + n;
        float z0 = 0.f, z1 = 0.f;
        if (b < a.n_b && j < n_p) {
            const double c = a.rot[2 * b], s = a.rot[2 * b + 1];
            const double2 u = reinterpret_cast<const double2*>(a.in)[(size_t)b * n_p + j];
            z0 = (float)(c * u.x + s * u.y);
            z1 = (float)(-s * u.x + c * u.y);
        }
        const int k = 2 * j;
        const int off = (n >> 3) * 8 * KP + (k >> 2) * 32 + (n & 7) * 4 + (k & 3);
        const float h0 = tf32_hi(z0), h1 = tf32_hi(z1);
        sB[off] = h0;
        sB[off + 1] = h1;
        sB[b_part + off] = z0 - h0;
        sB[b_part + off + 1] = z1 - h1;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (tid == 0) {
        const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_N >> 3) << 17) | ((128u >> 4) << 24);
        const uint32_t sA0 = smem_u32(sA), sB0 = smem_u32(sB);
        const uint32_t sbo_b = 32u * (uint32_t)KP;
        bool ok = true;
        int issued = KC < 2 ? KC : 2;  // chunks copied so far
        int consumed = 0;              // chunks whose copy has landed
        for (int c = 0; c < KC && ok; ++c) {
            const int s = c & 1;
            ok = mbar_wait(&bars[s], (c >> 1) & 1, a.err);
            if (!ok) break;
            consumed = c + 1;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int mt = 0; mt < MT; ++mt) {
                const uint32_t d = tmem + (uint32_t)(mt * TC_N);
                for (int kk = 0; kk < TC_KC / 8; ++kk) {
                    const int kg = c * (TC_KC / 8) + kk;  // global K step (8 columns)
                    const uint32_t a_hi = sA0 + (uint32_t)((s * stage_floats + (0 * MT + mt) * TC_TILE_FLOATS) * 4 + kk * 256);
                    const uint32_t a_lo = sA0 + (uint32_t)((s * stage_floats + (1 * MT + mt) * TC_TILE_FLOATS) * 4 + kk * 256);
                    const uint32_t z_hi = sB0 + (uint32_t)(kg * 256);
                    const uint32_t z_lo = sB0 + (uint32_t)(b_part * 4 + kg * 256);
                    const uint64_t dah = smem_desc(a_hi, 128, 1024), dal = smem_desc(a_lo, 128, 1024);
                    const uint64_t dzh = smem_desc(z_hi, 128, sbo_b), dzl = smem_desc(z_lo, 128, sbo_b);
                    mma_tf32(d, dah, dzh, idesc, (c | kk) ? 1 : 0);
                    mma_tf32(d, dah, dzl, idesc, 1);
                    mma_tf32(d, dal, dzh, idesc, 1);
                }
            }
            mma_commit(&bars[2 + s]);
            // refill the other stage (chunk c - 1's, whose products were issued before these)
            if (c >= 1 && c + 1 < KC && issued == c + 1) {
                const int s2 = (c + 1) & 1;
                ok = mbar_wait(&bars[2 + s2], ((c - 1) >> 1) & 1, a.err);
                if (!ok) break;
                mbar_expect_tx(&bars[s2], chunk_bytes);
                bulk_copy(sA + s2 * stage_floats, a.A + (size_t)(c + 1) * stage_floats, chunk_bytes, &bars[s2]);
                ++issued;
            }
        }
        mma_commit(&bars[4]);
        if (!ok) {
            // let the copies issued but not yet landed arrive before the CTA exits (bounded)
            for (int c = consumed; c < issued; ++c) mbar_wait(&bars[c & 1], (c >> 1) & 1, nullptr);
        }
    }
    __syncwarp();
    const bool landed = mbar_wait(&bars[4], 0, a.err);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // one decision for the whole CTA (the epilogue has block barriers)
    const bool good = __syncthreads_and(landed && !*a.err);

    if (good) {
        float acc[2][TC_N];
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
            if (mt < MT) tmem_ld16(tmem + lane_base + (uint32_t)(mt * TC_N), acc[mt]);
        if constexpr (MODE == TC_BODYFRAME) {
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                if (mt >= MT) break;
                const int m = mt * 128 + warp * 32 + lane;
                if (m < n2)
                    for (int n = 0; n < TC_N; ++n)
                        if (b0 + n < a.n_b) a.out_g[(size_t)(b0 + n) * n2 + m] = acc[mt][n];
            }
        } else if constexpr (MODE == TC_ROTATE) {
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                if (mt >= MT) break;
                const int m = mt * 128 + warp * 32 + lane;
                for (int n = 0; n < TC_N; ++n) {
                    const float other = __shfl_xor_sync(0xffffffffu, acc[mt][n], 1);
                    const int b = b0 + n;
                    if ((lane & 1) == 0 && m < n2 && b < a.n_b) {
                        const double c = a.rot[2 * b], s = a.rot[2 * b + 1];
                        const double gx = acc[mt][n], gy = other;
                        reinterpret_cast<double2*>(a.out)[(size_t)b * n_p + (m >> 1)] =
                            make_double2(c * gx - s * gy, s * gx + c * gy);
                    }
                }
            }
        } else {  // TC_PRECOND
            // K_ref^T g per body, as H^T z (M_ref^+ is symmetric, so K_ref^T M_ref^+ z = H^T z):
            // g carries large components along the near-null normal modes that K_ref^T
            // cancels, z and H do not, so H^T z keeps FP32 accuracy where K_ref^T g loses it
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                if (mt >= MT) break;
                const int m = mt * 128 + warp * 32 + lane;
                const bool row = m < n2;
                const float h0 = row ? a.H[m] : 0.f, h1 = row ? a.H[n2 + m] : 0.f, h2 = row ? a.H[2 * n2 + m] : 0.f;
                for (int n = 0; n < TC_N; ++n) {
                    // z (high + low part: the FP32 value) of body n at K index m
                    const int off = (n >> 3) * 8 * KP + (m >> 2) * 32 + (n & 7) * 4 + (m & 3);
                    const float z = row ? sB[off] + sB[b_part + off] : 0.f;
                    float sx = h0 * z, sy = h1 * z, st = h2 * z;
                    for (int o = 16; o > 0; o >>= 1) {
                        sx += __shfl_xor_sync(0xffffffffu, sx, o);
                        sy += __shfl_xor_sync(0xffffffffu, sy, o);
                        st += __shfl_xor_sync(0xffffffffu, st, o);
                    }
                    if (lane == 0) {
                        float* r = red + (mt * 4 + warp) * 48 + 3 * n;
                        r[0] = sx;
                        r[1] = sy;
                        r[2] = st;
                    }
                }
            }
            __syncthreads();
            if (tid < TC_N && b0 + tid < a.n_b) {
                const int b = b0 + tid;
                double tx = 0, ty = 0, tt = 0;
                for (int q = 0; q < 4 * MT; ++q) {
                    tx += red[q * 48 + 3 * tid];
                    ty += red[q * 48 + 3 * tid + 1];
                    tt += red[q * 48 + 3 * tid + 2];
                }
                const double c = a.rot[2 * b], s = a.rot[2 * b + 1];
                const double* rU = a.in + 2 * (size_t)a.n_b * n_p;
                const double ax = c * rU[3 * b] + s * rU[3 * b + 1] + tx;
                const double ay = -s * rU[3 * b] + c * rU[3 * b + 1] + ty;
                const double at = rU[3 * b + 2] + tt;
                const double u0 = -(a.nt[0] * ax + a.nt[1] * ay + a.nt[2] * at);
                const double u1 = -(a.nt[3] * ax + a.nt[4] * ay + a.nt[5] * at);
                const double u2 = -(a.nt[6] * ax + a.nt[7] * ay + a.nt[8] * at);
                Us[3 * tid] = u0;
                Us[3 * tid + 1] = u1;
                Us[3 * tid + 2] = u2;
                a.out_U[3 * b] = c * u0 - s * u1;
                a.out_U[3 * b + 1] = s * u0 + c * u1;
                a.out_U[3 * b + 2] = u2;
            }
            __syncthreads();
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                if (mt >= MT) break;
                const int m = mt * 128 + warp * 32 + lane;
                const bool row = m < n2;
                const float h0 = row ? a.H[m] : 0.f, h1 = row ? a.H[n2 + m] : 0.f, h2 = row ? a.H[2 * n2 + m] : 0.f;
                for (int n = 0; n < TC_N; ++n) {
                    const float v = acc[mt][n] + h0 * (float)Us[3 * n] + h1 * (float)Us[3 * n + 1] +
                                    h2 * (float)Us[3 * n + 2];
                    const float other = __shfl_xor_sync(0xffffffffu, v, 1);
                    const int b = b0 + n;
                    if ((lane & 1) == 0 && row && b < a.n_b) {
                        const float c = (float)a.rot[2 * b], s = (float)a.rot[2 * b + 1];
                        reinterpret_cast<double2*>(a.out)[(size_t)b * n_p + (m >> 1)] =
                            make_double2((double)(c * v - s * other), (double)(s * v + c * other));
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem));
}

size_t tc_smem_bytes(int KP, int MT) {
    return (size_t)2 * TC_N * KP * 4 + (size_t)2 * 2 * MT * TC_TILE_FLOATS * 4 + 5 * 8 + 16 + 4 * 2 * 48 * 4 +
           TC_N * 3 * 8;
}

uint32_t host_tf32_rna(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u += 0x1000u;
    u &= 0xFFFFE000u;
    return u;
}

}  // namespace

// Lay out B_ref (row-major n2 x n2, FP64) for k_block_tc: TF32 high and low parts in
// chunks of 32 K-columns, M-tiles of 128 rows, the operand layout of the file header.
fbim_status tc_prepare(fbim_handle_s* h, const std::vector<double>& Bref, int n2, TcBlock& out) {
    out = TcBlock();
    out.n2 = n2;
    out.KP = (n2 + TC_KC - 1) / TC_KC * TC_KC;
    out.MT = (n2 + 127) / 128;
    out.KC = out.KP / TC_KC;
    if (out.MT > 2) return FBIM_OK;  // not available: the caller keeps the library GEMM
    const size_t stage = (size_t)2 * out.MT * TC_TILE_FLOATS;
    std::vector<float> A(stage * out.KC, 0.f);
    for (int c = 0; c < out.KC; ++c)
        for (int p = 0; p < 2; ++p)
            for (int mt = 0; mt < out.MT; ++mt) {
                float* tile = A.data() + c * stage + (size_t)(p * out.MT + mt) * TC_TILE_FLOATS;
                for (int r = 0; r < 128; ++r)
                    for (int kk = 0; kk < TC_KC; ++kk) {
                        const int row = mt * 128 + r, k = c * TC_KC + kk;
                        const double v = (row < n2 && k < n2) ? Bref[(size_t)row * n2 + k] : 0.0;
                        const uint32_t hb = host_tf32_rna((float)v);
                        float hi;
                        std::memcpy(&hi, &hb, 4);
                        const float val = p == 0 ? hi : (float)(v - (double)hi);
                        tile[(r / 8) * 256 + (kk / 4) * 32 + (r % 8) * 4 + kk % 4] = val;
                    }
            }
    FBIM_CUDA_TRY(h, cudaMalloc(&out.A, A.size() * sizeof(float)));
    FBIM_CUDA_TRY(h, cudaMemcpy(out.A, A.data(), A.size() * sizeof(float), cudaMemcpyHostToDevice));
    // the kernels' limit is per kernel, not per handle: set it once to the largest
    // layout any handle can have (2 n_p = 256), so that handles of other sizes interleave
    const int smem = (int)tc_smem_bytes(256, 2);
    FBIM_CUDA_TRY(h, cudaFuncSetAttribute(k_block_tc<TC_ROTATE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    FBIM_CUDA_TRY(h, cudaFuncSetAttribute(k_block_tc<TC_BODYFRAME>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    FBIM_CUDA_TRY(h, cudaFuncSetAttribute(k_block_tc<TC_PRECOND>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    out.ready = true;
    return FBIM_OK;
}

fbim_status tc_check(fbim_handle_s* h) {
    Solver* S = h->solver;
    if (!S || !S->tc_err) return FBIM_OK;
    int e = 0;
    FBIM_CUDA_TRY(h, cudaMemcpyAsync(&e, S->tc_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    FBIM_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    if (e) {
        h->fail("a tensor-core block operator gave up a bounded wait (results of this call are invalid)");
        cudaMemsetAsync(S->tc_err, 0, sizeof(int), h->stream);
        return FBIM_ERR_TIMEOUT;
    }
    return FBIM_OK;
}

void tc_free(TcBlock& b) {
    cudaFree(b.A);
    b = TcBlock();
}

// Launch k_block_tc on the handle's stream.  mode: 0 rotate (out), 1 body frame
// (out_g), 2 preconditioner body solve (out = mu, out_U).
fbim_status tc_apply(fbim_handle_s* h, const TcBlock& B, int mode, const double* in, double* out, double* out_U,
                     float* out_g, const float* H, const double* Nt, int* err) {
    TcArgs a{};
    a.A = B.A;
    a.n_b = h->n_b;
    a.n_p = h->n_p;
    a.n2 = B.n2;
    a.KP = B.KP;
    a.MT = B.MT;
    a.KC = B.KC;
    a.rot = h->rot;
    a.in = in;
    a.ref = h->ref;
    a.H = H;
    if (Nt)
        for (int i = 0; i < 9; ++i) a.nt[i] = Nt[i];
    a.out = out;
    a.out_U = out_U;
    a.out_g = out_g;
    a.err = err;
    const unsigned grid = (unsigned)((h->n_b + TC_N - 1) / TC_N);
    const size_t smem = tc_smem_bytes(B.KP, B.MT);
    if (mode == TC_ROTATE)
        k_block_tc<TC_ROTATE><<<grid, 128, smem, h->stream>>>(a);
    else if (mode == TC_BODYFRAME)
        k_block_tc<TC_BODYFRAME><<<grid, 128, smem, h->stream>>>(a);
    else
        k_block_tc<TC_PRECOND><<<grid, 128, smem, h->stream>>>(a);
    h->launches += 1;
    FBIM_CUDA_TRY(h, cudaGetLastError());
    return FBIM_OK;
}

}  // namespace fbim
