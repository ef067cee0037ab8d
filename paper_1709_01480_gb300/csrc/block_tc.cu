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
// Tensor-core form.  tcgen05.mma kind::tf32, M = 128 rows of B_ref per CTA (a CTA
// per 128-row tile of B_ref and 16 bodies), N = 16 bodies, K = 8 per instruction,
// FP32 accumulators in tensor memory.  FP32 accuracy from TF32 operands by the
// three-term split a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi (a_hi = a rounded to TF32,
// a_lo = a - a_hi): the dropped a_lo b_lo and the TF32 truncation of the low parts are
// ~2^-20 relative (the high part is the value with its low 13 mantissa bits cleared).
// B_ref is laid out once, at setup, tile by tile in the operand layout below, in FP32,
// and streamed through shared memory in chunks of 32 K-columns by bulk copies with
// mbarrier completion, four chunks in flight; two warps split each chunk into its TF32
// parts as it lands.  The
// CTA's Z tile (16 bodies x all K) is formed in shared memory by its threads while
// the first chunks land.  The body solve needs K_ref^T g over all rows; it is formed
// as H^T z from the Z tile (M_ref^+ is symmetric), so the CTAs of the two row tiles
// of a body group need not exchange anything.
//
// Operand layout: K-major with the 128-byte swizzle, the tensor core's full-rate form.
// Per 32 K-columns (128 bytes of FP32), row r of an operand sits at (r/8) 1024 +
// (r%8) 128 bytes, its 16-byte chunk c at chunk position c ^ (r%8); the 8-row groups
// are 1024 bytes apart (stride byte offset), the atoms 1024-byte aligned, and the K
// steps of 8 columns inside an atom start 32 bytes apart.
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
constexpr int TC_STAGES = 4;                 // chunk stages: FP32 chunk (then its high part) + low part
// Independent accumulators, one per (K step within a chunk, split term): products that
// share an accumulator run one after another (each waits for the previous sum), so
// twelve chains of eight keep the tensor pipe busy where one chain of 96 left it idle.
constexpr int TC_ACC = 12;
constexpr int TC_TMEM_COLS = 256;            // TC_ACC x 16 columns, rounded to a power of 2
constexpr unsigned long long TC_WAIT_NS = 250000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Shared-memory matrix descriptor of a K-major operand with the 128-byte swizzle:
// start address, leading byte offset (unused by this layout: 16), stride byte offset
// 1024 (8 rows x 128 bytes), fixed field 0b001 at bits 46-48, layout 2 (128-byte
// swizzle) at bits 61-63.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)(16 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// float offset of element (row, k) in a K-major 128-byte-swizzled operand whose K
// atoms (32 columns) of all its rows are atom_floats apart
__device__ __host__ __forceinline__ int sw128_off(int row, int k, int atom_floats) {
    return (k >> 5) * atom_floats + (row >> 3) * 256 + (row & 7) * 32 + ((((k & 31) >> 2) ^ (row & 7)) << 2) +
           (k & 3);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, unsigned parity) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Bounded wait for the phase with the given parity; false (and *err set, err non-null)
// on expiry.  The global timer is read only once the phase is late, and then every
// 64 polls (each poll may itself suspend the thread for a while).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int* err) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (unsigned it = 1;; ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 63u) == 0u && globaltimer() - t0 > TC_WAIT_NS) {
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

// double -> float and float -> double by integer operations: GB300's FP64 pipe, which
// also runs the F2F conversions, is ~1/64 of its FP32 rate and was this kernel's
// bound.  d2f truncates the mantissa (within one float ulp of rounding) and flushes
// values below the float range to zero; f2d is exact for normal floats.  Inputs are
// finite (the solvers check for non-finite values).
__device__ __forceinline__ float d2f(double x) {
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7FFu) - 1023 + 127;
    if (e <= 0) return __uint_as_float(sign);
    if (e >= 255) return __uint_as_float(sign | 0x7F800000u);
    return __uint_as_float(sign | ((unsigned)e << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29));
}

__device__ __forceinline__ double f2d(float f) {
    const unsigned u = __float_as_uint(f), sign = u & 0x80000000u, e = (u >> 23) & 0xFFu;
    if (e == 0u) return __hiloint2double((int)sign, 0);
    return __hiloint2double((int)(sign | ((e - 127u + 1023u) << 20) | ((u & 0x7FFFFFu) >> 3)), (int)(u << 29));
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

// 8 consecutive accumulator columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

struct TcArgs {
    const float* A;       // B_ref in the operand layout [MT][KC][128 x 32], FP32
    int n_b, n_p, n2, KP, MT, KC;
    const double* rot;    // [n_b][2] (cos, sin)
    const double* in;     // [n_b * n_p][2] (then [n_b][3] r_U for TC_PRECOND)
    const double* ref;    // [n_p][2] reference nodes (TC_PRECOND)
    const float* H;       // [3][n2] M_ref^+ K_ref (TC_PRECOND)
    float ntf[9];         // N~_ref row-major (TC_PRECOND)
    double* out;          // [n_b * n_p][2] (TC_ROTATE: out; TC_PRECOND: mu)
    double* out_U;        // [n_b][3] (TC_PRECOND)
    float* out_g;         // [n_b][n2] (TC_BODYFRAME)
    int* err;             // failure flag
};

enum { TC_ROTATE = 0, TC_BODYFRAME = 1, TC_PRECOND = 2 };

// Roles of the 8 warps: all form the Z tile; then warp 0 lane 0 issues the products,
// warp 1 lane 0 refills the chunk stages, warps 2-3 split each landed FP32 chunk of
// B_ref into its TF32 high (in place) and low parts, and warps 4-7 (TC_PRECOND) form
// H^T z and the body solves; all read the accumulators out and write the results.
constexpr int TC_THREADS = 256;
constexpr int TC_SPLITTERS = 64;  // warps 2-3

template <int MODE>
__global__ void __launch_bounds__(TC_THREADS, 1) k_block_tc(TcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // the swizzle atoms need 1024-byte alignment in the shared window
    unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const int KP = a.KP, KC = a.KC, n2 = a.n2, n_p = a.n_p;
    const int mt = blockIdx.y;                    // this CTA's 128-row tile of B_ref
    const int NS = KC < TC_STAGES ? KC : TC_STAGES;
    // carve: Z tile (2 parts x 16 x KP floats), chunk stages (the FP32 chunk lands in the
    // high slot and is split in place), input slice, barriers, scratch
    float* sB = reinterpret_cast<float*>(smem);
    const int b_part = TC_N * KP;  // floats per part
    float* sA = sB + 2 * b_part;
    constexpr int stage_floats = 2 * TC_TILE_FLOATS;
    double2* sIn = reinterpret_cast<double2*>(sA + TC_STAGES * stage_floats);     // [16 n_p] input slice
    uint64_t* bars = reinterpret_cast<uint64_t*>(sIn + TC_N * (KP / 2));
    uint64_t* full = bars;                   // [S] chunk landed
    uint64_t* split = bars + TC_STAGES;      // [S] chunk split into its two parts
    uint64_t* empty = bars + 2 * TC_STAGES;  // [S] chunk's products done
    uint64_t* done = bars + 3 * TC_STAGES;   // all products done
    uint64_t* zin = done + 1;                // input slice landed
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(zin + 1);
    int* s_count = reinterpret_cast<int*>(tmem_slot + 1);                          // [2] split, issued
    float* red = reinterpret_cast<float*>(tmem_slot + 4);                           // [4 warps][48]
    float* Usf = red + 4 * 48;                                                     // [16][3] body velocities U'
    float2* sRot = reinterpret_cast<float2*>(Usf + TC_N * 3);                       // [16] (cos, sin)
    float* sRU = reinterpret_cast<float*>(sRot + TC_N);                            // [16][3] force residual
    float* sH = sRU + TC_N * 3 + 4;                                                // [3][KP] (TC_PRECOND)
    const int b0 = blockIdx.x * TC_N;
    const float* Atile = a.A + (size_t)mt * KC * TC_TILE_FLOATS;
    // an earlier launch failed: leave the outputs alone (one decision for the whole CTA)
    if (__syncthreads_or(tid == 0 ? *a.err : 0)) return;

    if (tid == 0) {
        for (int i = 0; i < TC_STAGES; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&split[i], TC_SPLITTERS);
            mbar_init(&empty[i], 1);
        }
        mbar_init(done, 1);
        mbar_init(zin, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_count[0] = 0;
        s_count[1] = 0;
    }
    // the CTA's rotations, force residuals and H (body solve), once, into shared memory
    if (tid < TC_N) {
        const int b = b0 + tid;
        const bool ok = b < a.n_b;
        sRot[tid] = ok ? make_float2(d2f(a.rot[2 * b]), d2f(a.rot[2 * b + 1])) : make_float2(1.f, 0.f);
        if (MODE == TC_PRECOND) {
            const double* rU = a.in + 2 * (size_t)a.n_b * n_p + 3 * (size_t)b;
            for (int q = 0; q < 3; ++q) sRU[3 * tid + q] = ok ? d2f(rU[q]) : 0.f;
        }
    }
    if constexpr (MODE == TC_PRECOND) {
        // 3 KP <= 768 entries: all loads of a thread issued before its stores
        float hv[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const int i = tid + r * TC_THREADS, c = i / KP, k = i - c * KP;
            hv[r] = (i < 3 * KP && k < n2) ? a.H[c * n2 + k] : 0.f;
        }
#pragma unroll
        for (int r = 0; r < 3; ++r)
            if (tid + r * TC_THREADS < 3 * KP) sH[tid + r * TC_THREADS] = hv[r];
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "n"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    __syncthreads();
    constexpr unsigned chunk_bytes = (unsigned)(TC_TILE_FLOATS * sizeof(float));  // FP32 chunk
    const int nb_cta = min(TC_N, a.n_b - b0);  // bodies of this CTA (the last one may be ragged)
    if (tid == 0) {  // the CTA's input slice (one contiguous run), then the first NS chunks of the tile
        const unsigned in_bytes = (unsigned)(nb_cta * n_p * 16);
        mbar_expect_tx(zin, in_bytes);
        bulk_copy(sIn, reinterpret_cast<const double2*>(a.in) + (size_t)b0 * n_p, in_bytes, zin);
        for (int c = 0; c < NS; ++c) {
            mbar_expect_tx(&full[c], chunk_bytes);
            bulk_copy(sA + c * stage_floats, Atile + (size_t)c * TC_TILE_FLOATS, chunk_bytes, &full[c]);
        }
    }
    // Z tile: z = R_b^T in_b for the CTA's bodies, split into TF32 high and low parts, each
    // part a 16-row K-major swizzled operand (K atoms 16 x 32 floats apart).  Half-warp h
    // takes body n and 16 consecutive nodes: its loads are one 256-byte run, and the two
    // half-warps of a warp (bodies n and n + 1) store to distinct banks through the swizzle.
    const bool in_ok = __syncthreads_and(mbar_wait(zin, 0, a.err));
    {
        const int h = tid >> 4, l = tid & 15;
        const int n_units = TC_N * (KP / 32);  // (body, 16-node block) pairs
#pragma unroll 2
        for (int u = h; u < n_units; u += TC_THREADS / 16) {
            const int n = u % TC_N, j = (u / TC_N) * 16 + l;
            float z0 = 0.f, z1 = 0.f;
            if (n < nb_cta && in_ok && j < n_p) {
                const double2 v = sIn[n * n_p + j];
                const float ux = d2f(v.x), uy = d2f(v.y), c = sRot[n].x, sn = sRot[n].y;
                z0 = fmaf(c, ux, sn * uy);
                z1 = fmaf(-sn, ux, c * uy);
            }
            const int off = sw128_off(n, 2 * j, TC_N * 32);
            const float h0 = tf32_hi(z0), h1 = tf32_hi(z1);
            sB[off] = h0;
            sB[off + 1] = h1;
            sB[b_part + off] = z0 - h0;
            sB[b_part + off + 1] = z1 - h1;
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (tid == 0) {  // MMA issue: one thread; never waits for the products it issued
        const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_N >> 3) << 17) | ((128u >> 4) << 24);
        // descriptors at the first stage and the Z tile's first atom; the others differ only
        // in the start-address field (16-byte units, no carry out of its 14 bits in 227 KB)
        const uint64_t dA0 = smem_desc_sw128(smem_u32(sA));
        const uint64_t dZ0 = smem_desc_sw128(smem_u32(sB));
        constexpr uint64_t lo_a = (uint64_t)(TC_TILE_FLOATS * 4) >> 4;   // A's low part
        const uint64_t lo_z = (uint64_t)(b_part * 4) >> 4;              // Z's low part
        for (int c = 0; c < KC; ++c) {
            const int s = c % NS;
            if (!mbar_wait(&split[s], (unsigned)(c / NS) & 1u, a.err)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // chunk c is one K atom: the A tile at its stage, the Z tile's atom c; K step kk
            // starts 32 bytes into the atom
            const uint64_t dah = dA0 + (uint64_t)(s * stage_floats * 4 >> 4);
            const uint64_t dzh = dZ0 + (uint64_t)(c * TC_N * 32 * 4 >> 4);
#pragma unroll
            for (int kk = 0; kk < TC_KC / 8; ++kk) {
                const uint64_t ka = (uint64_t)(kk * 32 >> 4);
                const uint32_t d = tmem + (uint32_t)(3 * kk * TC_N);  // accumulators 3 kk .. 3 kk + 2
                mma_tf32(d, dah + ka, dzh + ka, idesc, c);
                mma_tf32(d + TC_N, dah + ka, dzh + lo_z + ka, idesc, c);
                mma_tf32(d + 2 * TC_N, dah + lo_a + ka, dzh + ka, idesc, c);
            }
            mma_commit(&empty[s]);  // the stage is free once these products are done
        }
        mma_commit(done);
    } else if (tid == 32) {  // refills: chunk c into the stage of chunk c - NS once that one is consumed
        int issued = NS;
        for (int c = NS; c < KC; ++c) {
            const int s = c % NS;
            if (!mbar_wait(&empty[s], (unsigned)((c - NS) / NS) & 1u, a.err)) break;
            mbar_expect_tx(&full[s], chunk_bytes);
            bulk_copy(sA + s * stage_floats, Atile + (size_t)c * TC_TILE_FLOATS, chunk_bytes, &full[s]);
            issued = c + 1;
        }
        s_count[1] = issued;
    } else if (warp == 2 || warp == 3) {
        // split each landed chunk: x -> high part (x with its low 13 mantissa bits cleared,
        // in place) + low part (the exact remainder), float4 at a time
        const int t = tid - 64;
        int split_n = 0;
        for (int c = 0; c < KC; ++c) {
            const int s = c % NS;
            if (!mbar_wait(&full[s], (unsigned)(c / NS) & 1u, a.err)) break;
            float4* hi = reinterpret_cast<float4*>(sA + s * stage_floats);
            float4* lo = hi + TC_TILE_FLOATS / 4;
#pragma unroll 4
            for (int i = t; i < TC_TILE_FLOATS / 4; i += TC_SPLITTERS) {
                const float4 x = hi[i];
                const float4 h = make_float4(__uint_as_float(__float_as_uint(x.x) & 0xFFFFE000u),
                                             __uint_as_float(__float_as_uint(x.y) & 0xFFFFE000u),
                                             __uint_as_float(__float_as_uint(x.z) & 0xFFFFE000u),
                                             __uint_as_float(__float_as_uint(x.w) & 0xFFFFE000u));
                hi[i] = h;
                lo[i] = make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&split[s])) : "memory");
            split_n = c + 1;
        }
        if (t == 0) s_count[0] = split_n;
    } else if (MODE == TC_PRECOND && warp >= 4) {
        // While the products run: K_ref^T g per body as H^T z (M_ref^+ is symmetric, so
        // K_ref^T M_ref^+ z = H^T z; g carries large components along the near-null normal
        // modes that K_ref^T cancels, z and H do not, so H^T z keeps FP32 accuracy where
        // K_ref^T g loses it), then the 3 x 3 body solves (FP32: the preconditioner's
        // precision).  Thread (n = lane % 16, k = 2 (warp - 4) + lane / 16 + 8 i).
        const int n = lane & 15;
        float sx = 0.f, sy = 0.f, st = 0.f;
        for (int k = 2 * (warp - 4) + (lane >> 4); k < n2; k += 8) {
            const int off = sw128_off(n, k, TC_N * 32);
            const float z = sB[off] + sB[b_part + off];  // the FP32 value
            sx = fmaf(sH[k], z, sx);
            sy = fmaf(sH[KP + k], z, sy);
            st = fmaf(sH[2 * KP + k], z, st);
        }
        sx += __shfl_xor_sync(0xffffffffu, sx, 16);
        sy += __shfl_xor_sync(0xffffffffu, sy, 16);
        st += __shfl_xor_sync(0xffffffffu, st, 16);
        if (lane < 16) {
            red[(warp - 4) * 48 + 3 * n] = sx;
            red[(warp - 4) * 48 + 3 * n + 1] = sy;
            red[(warp - 4) * 48 + 3 * n + 2] = st;
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");  // warps 4 to 7 only
        if (warp == 4 && lane < TC_N && lane < nb_cta) {
            const int b = b0 + lane;
            const float tx = red[3 * lane] + red[48 + 3 * lane] + red[96 + 3 * lane] + red[144 + 3 * lane];
            const float ty = red[3 * lane + 1] + red[48 + 3 * lane + 1] + red[96 + 3 * lane + 1] + red[144 + 3 * lane + 1];
            const float tt = red[3 * lane + 2] + red[48 + 3 * lane + 2] + red[96 + 3 * lane + 2] + red[144 + 3 * lane + 2];
            const float c = sRot[lane].x, s = sRot[lane].y;
            const float r0 = sRU[3 * lane], r1 = sRU[3 * lane + 1], r2 = sRU[3 * lane + 2];
            const float ax = fmaf(c, r0, fmaf(s, r1, tx));
            const float ay = fmaf(-s, r0, fmaf(c, r1, ty));
            const float at = r2 + tt;
            const float u0 = -(a.ntf[0] * ax + a.ntf[1] * ay + a.ntf[2] * at);
            const float u1 = -(a.ntf[3] * ax + a.ntf[4] * ay + a.ntf[5] * at);
            const float u2 = -(a.ntf[6] * ax + a.ntf[7] * ay + a.ntf[8] * at);
            Usf[3 * lane] = u0;
            Usf[3 * lane + 1] = u1;
            Usf[3 * lane + 2] = u2;
            if (mt == 0) {
                a.out_U[3 * b] = f2d(fmaf(c, u0, -s * u1));
                a.out_U[3 * b + 1] = f2d(fmaf(s, u0, c * u1));
                a.out_U[3 * b + 2] = f2d(u2);
            }
        }
    }
    __syncwarp();
    const bool landed = mbar_wait(done, 0, a.err);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // one decision for the whole CTA (the epilogue has block barriers)
    const bool good = __syncthreads_and(landed && !*a.err);
    if (!good && tid == 0) {
        // products and copies still in flight finish before the CTA frees its memory (bounded)
        mbar_wait(done, 0, nullptr);
        if (!in_ok) mbar_wait(zin, 0, nullptr);
        for (int c = s_count[0]; c < s_count[1]; ++c) mbar_wait(&full[c % NS], (unsigned)(c / NS) & 1u, nullptr);
    }

    if (good) {
        // warp w reads rows 32 (w % 4) .. + 31 (its lane quarter) for the bodies of half
        // w / 4, and sums the accumulators
        const int hb = warp >> 2;  // body half: n = 8 hb .. 8 hb + 7
        float acc[8];
        {
            const uint32_t tl = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(8 * hb);
            tmem_ld8(tl, acc);
#pragma unroll
            for (int q = 1; q < TC_ACC; ++q) {
                float t[8];
                tmem_ld8(tl + (uint32_t)(q * TC_N), t);
#pragma unroll
                for (int i = 0; i < 8; ++i) acc[i] += t[i];
            }
        }
        const int m = mt * 128 + (warp & 3) * 32 + lane;  // this thread's row of the tile
        const bool row = m < n2;
        if constexpr (MODE == TC_BODYFRAME) {
            if (row)
                for (int i = 0; i < 8; ++i)
                    if (b0 + 8 * hb + i < a.n_b) a.out_g[(size_t)(b0 + 8 * hb + i) * n2 + m] = acc[i];
        } else if constexpr (MODE == TC_ROTATE) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int n = 8 * hb + i;
                const float other = __shfl_xor_sync(0xffffffffu, acc[i], 1);
                const int b = b0 + n;
                if ((lane & 1) == 0 && row && b < a.n_b) {
                    const float c = sRot[n].x, s = sRot[n].y, gx = acc[i], gy = other;
                    reinterpret_cast<double2*>(a.out)[(size_t)b * n_p + (m >> 1)] =
                        make_double2(f2d(fmaf(c, gx, -s * gy)), f2d(fmaf(s, gx, c * gy)));
                }
            }
        } else {  // TC_PRECOND: mu = R (g + H U') with U' from the body solves above
            const float h0 = row ? sH[m] : 0.f, h1 = row ? sH[KP + m] : 0.f, h2 = row ? sH[2 * KP + m] : 0.f;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int n = 8 * hb + i;
                const float v = fmaf(h0, Usf[3 * n], fmaf(h1, Usf[3 * n + 1], fmaf(h2, Usf[3 * n + 2], acc[i])));
                const float other = __shfl_xor_sync(0xffffffffu, v, 1);
                const int b = b0 + n;
                if ((lane & 1) == 0 && row && b < a.n_b) {
                    const float c = sRot[n].x, s = sRot[n].y;
                    reinterpret_cast<double2*>(a.out)[(size_t)b * n_p + (m >> 1)] =
                        make_double2(f2d(fmaf(c, v, -s * other)), f2d(fmaf(s, v, c * other)));
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(TC_TMEM_COLS));
}

// the carve of k_block_tc: Z tile, chunk stages, input slice, barriers, TMEM slot, warp
// sums, U', rotations, force residuals, H
size_t tc_smem_bytes(int KP) {
    return 1024 + (size_t)2 * TC_N * KP * 4 + (size_t)TC_STAGES * 2 * TC_TILE_FLOATS * 4 + (size_t)TC_N * (KP / 2) * 16 +
           (3 * TC_STAGES + 2) * 8 + 16 + 4 * 48 * 4 + TC_N * 3 * 4 + TC_N * 8 + TC_N * 3 * 4 + 16 + (size_t)3 * KP * 4;
}


}  // namespace

// Lay out B_ref (row-major n2 x n2, FP64) for k_block_tc: per 128-row tile, per chunk of
// 32 K-columns (one swizzle atom), its FP32 values in the operand layout of the file
// header (the kernel splits them into TF32 parts as they land).
fbim_status tc_prepare(fbim_handle_s* h, const std::vector<double>& Bref, int n2, TcBlock& out) {
    out = TcBlock();
    out.n2 = n2;
    out.KP = (n2 + TC_KC - 1) / TC_KC * TC_KC;
    out.MT = (n2 + 127) / 128;
    out.KC = out.KP / TC_KC;
    if (out.MT > 2) return FBIM_OK;  // not available: the caller keeps the library GEMM
    std::vector<float> A((size_t)TC_TILE_FLOATS * out.KC * out.MT, 0.f);
    for (int mt = 0; mt < out.MT; ++mt)
        for (int c = 0; c < out.KC; ++c) {
            float* tile = A.data() + ((size_t)mt * out.KC + c) * TC_TILE_FLOATS;
            for (int r = 0; r < 128; ++r)
                for (int kk = 0; kk < TC_KC; ++kk) {
                    const int row = mt * 128 + r, k = c * TC_KC + kk;
                    tile[sw128_off(r, kk, 0)] = (row < n2 && k < n2) ? (float)Bref[(size_t)row * n2 + k] : 0.f;
                }
        }
    FBIM_CUDA_TRY(h, cudaMalloc(&out.A, A.size() * sizeof(float)));
    FBIM_CUDA_TRY(h, cudaMemcpy(out.A, A.data(), A.size() * sizeof(float), cudaMemcpyHostToDevice));
    // the kernels' limit is per kernel, not per handle: set it once to the largest
    // layout any handle can have (2 n_p = 256), so that handles of other sizes interleave
    const int smem = (int)tc_smem_bytes(256);
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
        for (int i = 0; i < 9; ++i) a.ntf[i] = (float)Nt[i];
    a.out = out;
    a.out_U = out_U;
    a.out_g = out_g;
    a.err = err;
    const dim3 grid((unsigned)((h->n_b + TC_N - 1) / TC_N), (unsigned)B.MT);
    const size_t smem = tc_smem_bytes(B.KP);
    if (mode == TC_ROTATE)
        k_block_tc<TC_ROTATE><<<grid, TC_THREADS, smem, h->stream>>>(a);
    else if (mode == TC_BODYFRAME)
        k_block_tc<TC_BODYFRAME><<<grid, TC_THREADS, smem, h->stream>>>(a);
    else
        k_block_tc<TC_PRECOND><<<grid, TC_THREADS, smem, h->stream>>>(a);
    h->launches += 1;
    FBIM_CUDA_TRY(h, cudaGetLastError());
    return FBIM_OK;
}

}  // namespace fbim
