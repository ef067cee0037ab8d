// Node geometry and the cell list (Sec. 3.1 node placement; Sec. 3.2 cell list).
//
// x_{beta,j} = q_beta + R(theta_beta) gamma_ref(s_j), wrapped into [0, L).
// Cells are n_box x n_box squares of side r_c = L / n_box; nodes are counted
// per cell, the counts scanned, the nodes scattered, and each cell's slots
// sorted by node index so that the cell-sorted order (and every sum over it)
// is deterministic.
#include "fbim_internal.h"

namespace fbim {

namespace {

__global__ void k_nodes(int N, int n_p, const double* __restrict__ Q, const double* __restrict__ ref, double L,
                        double r_c, int n_box, double* __restrict__ x, int* __restrict__ cell,
                        int* __restrict__ count, int* __restrict__ flags) {
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

}  // namespace

fbim_status build_geometry(fbim_handle_s* h) {
    const int N = h->N, nc = h->n_cell();
    FBIM_CUDA_TRY(h, cudaMemsetAsync(h->cell_fill, 0, sizeof(int) * nc, h->stream));
    const int tb = 256;
    k_nodes<<<(N + tb - 1) / tb, tb, 0, h->stream>>>(N, h->n_p, h->Q, h->ref, h->L, h->r_c, h->n_box, h->x, h->cell,
                                                     h->cell_fill, h->flags);
    k_scan<<<1, 1024, 0, h->stream>>>(nc, h->cell_fill, h->cell_start);
    FBIM_CUDA_TRY(h, cudaMemsetAsync(h->cell_fill, 0, sizeof(int) * nc, h->stream));
    k_scatter<<<(N + tb - 1) / tb, tb, 0, h->stream>>>(N, h->cell, h->cell_start, h->cell_fill, h->perm);
    k_sort_cells<<<(nc + tb - 1) / tb, tb, 0, h->stream>>>(nc, h->cell_start, h->perm, h->slot);
    FBIM_CUDA_TRY(h, cudaGetLastError());
    if (h->e64.ready) FBIM_TRY(refresh_offsets<double>(h));
    if (h->e32.ready) FBIM_TRY(refresh_offsets<float>(h));
    return FBIM_OK;
}

}  // namespace fbim
