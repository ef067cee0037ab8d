// Node geometry and the cell list (Sec. 3.1 node placement; Sec. 3.2 cell list).
//
// x_{beta,j} = q_beta + R(theta_beta) gamma_ref(s_j), wrapped into [0, L).
// Cells are n_box x n_box squares of side r_c = L / n_box; nodes are counted
// per cell, the counts scanned, the nodes scattered, and each cell's slots
// sorted by node index so that the cell-sorted order (and every sum over it)
// is deterministic.  The same counting sort orders the nodes by the grid tile
// of their nearest grid point, the layout of the wave-space kernels.
#include "fbim_internal.h"

namespace fbim {

namespace {

__global__ void k_nodes(int N, int n_p, const double* __restrict__ Q, const double* __restrict__ ref, double L,
                        double r_c, int n_box, double hgrid, int M, int TS, int n_tile, double* __restrict__ x,
                        int* __restrict__ cell, int* __restrict__ count, int2* __restrict__ gbase,
                        int* __restrict__ tcount, int* __restrict__ flags) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= N) return;
    int b = m / n_p, j = m - b * n_p;
    double qx = Q[3 * b], qy = Q[3 * b + 1], th = Q[3 * b + 2];
    double c, s;
    sincos(th, &s, &c);
    double gx = ref[2 * j], gy = ref[2 * j + 1];
    double px = qx + c * gx - s * gy;
    double py = qy + s * gx + c * gy;
    if (!isfinite(px) || !isfinite(py)) {
        atomicOr(&flags[0], 1);
        px = 0.0;
        py = 0.0;
    }
    px -= L * floor(px / L);
    py -= L * floor(py / L);
    if (px >= L) px -= L;
    if (py >= L) py -= L;
    x[2 * m] = px;
    x[2 * m + 1] = py;
    int cx = min((int)(px / r_c), n_box - 1);
    int cy = min((int)(py / r_c), n_box - 1);
    int cid = cy * n_box + cx;
    cell[m] = cid;
    atomicAdd(&count[cid], 1);
    // nearest grid point and its wave-space tile
    int bx = ((int)rint(px / hgrid)) % M, by = ((int)rint(py / hgrid)) % M;
    gbase[m] = make_int2(bx, by);
    atomicAdd(&tcount[(by / TS) * n_tile + bx / TS], 1);
}

// Exclusive scan of count[0..n) into start[0..n], one block, any n.
__global__ void k_scan(int n, const int* __restrict__ count, int* __restrict__ start) {
    __shared__ int part[1024];
    int tid = threadIdx.x;
    int per = (n + blockDim.x - 1) / blockDim.x;
    int lo = min(n, tid * per), hi = min(n, lo + per);
    int s = 0;
    for (int i = lo; i < hi; ++i) s += count[i];
    part[tid] = s;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        int v = tid >= off ? part[tid - off] : 0;
        __syncthreads();
        part[tid] += v;
        __syncthreads();
    }
    int run = tid > 0 ? part[tid - 1] : 0;
    for (int i = lo; i < hi; ++i) {
        start[i] = run;
        run += count[i];
    }
    if (tid == blockDim.x - 1) start[n] = part[tid];
}

__global__ void k_scatter(int N, const int* __restrict__ cell, const int* __restrict__ start, int* __restrict__ fill,
                          int* __restrict__ perm) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= N) return;
    int c = cell[m];
    int pos = start[c] + atomicAdd(&fill[c], 1);
    perm[pos] = m;
}

__global__ void k_scatter_slots(int N, const int* __restrict__ key, const int* __restrict__ start,
                                int* __restrict__ fill, int* __restrict__ perm, int* __restrict__ slot) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= N) return;
    int c = key[m];
    int pos = start[c] + atomicAdd(&fill[c], 1);
    perm[pos] = m;
    slot[m] = pos;
}

__global__ void k_sort_cells(int n_cell, const int* __restrict__ start, int* __restrict__ perm,
                             int* __restrict__ slot) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cell) return;
    int lo = start[c], hi = start[c + 1];
    for (int i = lo + 1; i < hi; ++i) {
        int key = perm[i];
        int k = i - 1;
        while (k >= lo && perm[k] > key) {
            perm[k + 1] = perm[k];
            --k;
        }
        perm[k + 1] = key;
    }
    for (int i = lo; i < hi; ++i) slot[perm[i]] = i;
}

__global__ void k_tile_of(int N, const int2* __restrict__ gbase, int TS, int n_tile, int* __restrict__ tile) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= N) return;
    int2 b = gbase[m];
    tile[m] = (b.y / TS) * n_tile + b.x / TS;
}

__global__ void k_rot(int n_b, const double* __restrict__ Q, double* __restrict__ rot) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_b) return;
    double c, s;
    sincos(Q[3 * b + 2], &s, &c);
    rot[2 * b] = c;
    rot[2 * b + 1] = s;
}

// Block-local exclusive scan of 1024 elements per block (256 threads x 4); the
// block total goes to totals[block].
__global__ void k_scan_local(int n, const int* __restrict__ in, int* __restrict__ out, int* __restrict__ totals) {
    __shared__ int warp_sum[8];
    const int base = blockIdx.x * 1024 + threadIdx.x * 4;
    int v[4], s = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        v[i] = (base + i < n) ? in[base + i] : 0;
        s += v[i];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = s;
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_sum[warp] = incl;
    __syncthreads();
    int before = 0, tot = 0;
    for (int w = 0; w < 8; ++w) {
        before += (w < warp) ? warp_sum[w] : 0;
        tot += warp_sum[w];
    }
    int run = before + incl - s;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
    if (threadIdx.x == 0) totals[blockIdx.x] = tot;
}

__global__ void k_scan_add(int n, int* __restrict__ out, const int* __restrict__ offs) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += offs[i / 1024];
}

}  // namespace

// out[0..n] = exclusive prefix sums of in[0..n) with out[n] the total.  Uses
// out[n + 1 ..] as scratch: out must hold n + 2 + 2 ceil(n / 1024) ints.
void scan_exclusive(cudaStream_t st, const int* in, int n, int* out) {
    const int nb = (n + 1023) / 1024;
    int* totals = out + n + 1;
    int* offs = totals + nb;
    k_scan_local<<<nb, 256, 0, st>>>(n, in, out, totals);
    k_scan<<<1, 1024, 0, st>>>(nb, totals, offs);  // offs[0..nb], offs[nb] = grand total
    k_scan_add<<<(n + 255) / 256, 256, 0, st>>>(n, out, offs);
    // out[n] = grand total
    cudaMemcpyAsync(out + n, offs + nb, sizeof(int), cudaMemcpyDeviceToDevice, st);
}

size_t scan_storage(int n) { return (size_t)n + 2 + 2 * (size_t)((n + 1023) / 1024); }

fbim_status build_geometry(fbim_handle_s* h) {
    const int N = h->N, nc = h->n_cell(), nt = h->n_tile * h->n_tile;
    ++h->geom_version;
    // flags 0 (non-finite coordinates) and 1 (coincident nodes) describe this geometry
    FBIM_CUDA_TRY(h, cudaMemsetAsync(h->flags, 0, 2 * sizeof(int), h->stream));
    FBIM_CUDA_TRY(h, cudaMemsetAsync(h->cell_fill, 0, sizeof(int) * nc, h->stream));
    FBIM_CUDA_TRY(h, cudaMemsetAsync(h->tile_fill, 0, sizeof(int) * nt, h->stream));
    const int tb = 256;
    k_nodes<<<(N + tb - 1) / tb, tb, 0, h->stream>>>(N, h->n_p, h->Q, h->ref, h->L, h->r_c, h->n_box, h->h, h->M,
                                                     h->TS, h->n_tile, h->x, h->cell, h->cell_fill, h->gbase,
                                                     h->tile_fill, h->flags);
    // cell list (real space)
    scan_exclusive(h->stream, h->cell_fill, nc, h->cell_start);
    FBIM_CUDA_TRY(h, cudaMemsetAsync(h->cell_fill, 0, sizeof(int) * nc, h->stream));
    k_scatter<<<(N + tb - 1) / tb, tb, 0, h->stream>>>(N, h->cell, h->cell_start, h->cell_fill, h->perm);
    k_sort_cells<<<(nc + tb - 1) / tb, tb, 0, h->stream>>>(nc, h->cell_start, h->perm, h->slot);
    // grid tiles (wave space): nodes sorted by the TS x TS tile holding their nearest grid point
    scan_exclusive(h->stream, h->tile_fill, nt, h->tile_start);
    FBIM_CUDA_TRY(h, cudaMemsetAsync(h->tile_fill, 0, sizeof(int) * nt, h->stream));
    k_tile_of<<<(N + tb - 1) / tb, tb, 0, h->stream>>>(N, h->gbase, h->TS, h->n_tile, h->tile_tmp);
    // (order inside a tile is left as scattered: wave-space sums do not depend on it
    // beyond the rounding of the shared-memory accumulation)
    k_scatter_slots<<<(N + tb - 1) / tb, tb, 0, h->stream>>>(N, h->tile_tmp, h->tile_start, h->tile_fill, h->tperm,
                                                             h->tslot);
    k_rot<<<(h->n_b + tb - 1) / tb, tb, 0, h->stream>>>(h->n_b, h->Q, h->rot);
    h->launches += 8;
    FBIM_CUDA_TRY(h, cudaGetLastError());
    // FP32 first: an FP32 handle's FP64 list is derived from its FP32 list
    if (h->e32.ready) FBIM_TRY(refresh_offsets<float>(h));
    if (h->e64.ready) FBIM_TRY(refresh_offsets<double>(h));
    return FBIM_OK;
}

fbim_status update_positions(fbim_handle_s* h, const double* Q_dev) {
    if (Q_dev != h->Q)
        FBIM_CUDA_TRY(h, cudaMemcpyAsync(h->Q, Q_dev, 3 * h->n_b * sizeof(double), cudaMemcpyDeviceToDevice,
                                         h->stream));
    return build_geometry(h);
}

namespace {
__global__ void k_differs(int n, const double* __restrict__ a, const double* __restrict__ b, int* __restrict__ flag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && __double_as_longlong(a[i]) != __double_as_longlong(b[i])) atomicOr(flag, 1);
}
}  // namespace

fbim_status update_positions_if_moved(fbim_handle_s* h, const double* Q_dev) {
    if (Q_dev == h->Q) return update_positions(h, Q_dev);
    const int n = 3 * h->n_b;
    FBIM_CUDA_TRY(h, cudaMemsetAsync(h->flags + 3, 0, sizeof(int), h->stream));
    k_differs<<<(n + 255) / 256, 256, 0, h->stream>>>(n, Q_dev, h->Q, h->flags + 3);
    h->launches += 1;
    int moved = 1;
    FBIM_CUDA_TRY(h, cudaMemcpyAsync(&moved, h->flags + 3, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    FBIM_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return moved ? update_positions(h, Q_dev) : FBIM_OK;
}

}  // namespace fbim
