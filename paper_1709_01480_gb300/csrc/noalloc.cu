// fbim_apply_real_noalloc: the real-space operator v = (M(t) + M(a)_sym) mu of an
// existing handle, computed without allocating device memory.
//
// Some callers cannot call cudaMalloc once they are running: a host that hands
// all device memory to its own pool at start-up, or a time-critical loop where
// an allocation could block or fail at an arbitrary moment.  fbim_apply_real may
// allocate on its first use of a precision; this variant never does.  Its
// scratch (the forces and the velocities in cell-sorted order) lives in a
// file-scope device array of fixed size, and the pair sum is evaluated on the
// fly from the handle's cell list instead of from a stored pair list.
//
// The array holds 2 x FBIM_NOALLOC_MAX_NODES double2 values (4 MiB) on every
// device that loads the library, for the life of the process.  All calls share
// it and it keeps the last call's contents; every entry a call reads is first
// written by the same call, so nothing needs clearing.  Calls whose work
// overlaps on the GPU (different streams, or different handles on one device)
// race on the array and must be serialised by the caller.
//
// Under CUDA's lazy module loading a module, and each kernel in it, is loaded
// (and its device memory allocated) when it is first used.  fbim_setup therefore
// runs noalloc_prepare on the handle's device: it looks up the array's address and
// launches each kernel of this file once on an empty range, so that the module,
// the kernels' code and their local memory are in place before the entry point is
// first called; the entry point itself then neither loads nor allocates.
#include <mutex>

#include "ewald_types.cuh"
#include "fbim_internal.h"

#define FBIM_NOALLOC_MAX_NODES 131072
#define FBIM_NOALLOC_MAX_DEVICES 64

namespace {

static __device__ __align__(256) double2 g_noalloc_scratch[2 * FBIM_NOALLOC_MAX_NODES];

// Host-side device address of g_noalloc_scratch per device ordinal.  The name of
// the array in host code is only a stand-in for the symbol, not a device address.
double2* g_scratch_addr[FBIM_NOALLOC_MAX_DEVICES] = {};
std::mutex g_scratch_lock;

__global__ void k_na_gather(int N, const int* __restrict__ perm, const double2* __restrict__ mu,
                            double2* __restrict__ mu_s) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < N) mu_s[s] = mu[perm[s]];
}

// Coincident nodes (r = 0) contribute nothing and raise flags[1], as in the pair-list
// build; fbim_setup and fbim_update_config report that flag as FBIM_ERR_OVERLAP.
__global__ void __launch_bounds__(128) k_na_pairs(int N, int n_box, double r_c, double rc2, double xi2, double pref,
                                                 fbim::ChebE1<double> ce, const int* __restrict__ perm,
                                                 const int* __restrict__ cell, const int* __restrict__ start,
                                                 const double2* __restrict__ off, const double2* __restrict__ mu_s,
                                                 double2* __restrict__ v_s, int* __restrict__ flags) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N) return;
    double ax = 0, ay = 0;
    fbim::for_each_pair<double>(t, n_box, r_c, rc2, perm, cell, start, off, [&](int s, double rx, double ry, double r2) {
        if (r2 == 0.0) {
            atomicOr(&flags[1], 1);
            return;
        }
        double z = xi2 * r2;
        double a = fbim::kernel_a<double>(ce, z);
        double b = exp(-z) / r2;
        double2 m = mu_s[s];
        double rm = rx * m.x + ry * m.y;
        ax += a * m.x + b * rx * rm;
        ay += a * m.y + b * ry * rm;
    });
    v_s[t] = make_double2(pref * ax, pref * ay);
}

__global__ void k_na_finish(int N, int n_p, int band, const int* __restrict__ slot, const double2* __restrict__ v_s,
                            const double* __restrict__ rot, const double* __restrict__ A,
                            const double2* __restrict__ mu, double2* __restrict__ v) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= N) return;
    double2 w = v_s[slot[m]];
    int b = m / n_p, j = m - b * n_p;
    double c = rot[2 * b], s = rot[2 * b + 1];
    double ax = 0, ay = 0;
    const int B = 2 * band + 1;
    for (int o = -band; o <= band; ++o) {
        int jj = j + o;
        jj += (jj < 0) ? n_p : 0;
        jj -= (jj >= n_p) ? n_p : 0;
        double2 u = mu[b * n_p + jj];
        double rx = c * u.x + s * u.y, ry = -s * u.x + c * u.y;  // R^T u
        const double* a = A + ((size_t)j * B + (o + band)) * 4;
        ax += a[0] * rx + a[1] * ry;
        ay += a[2] * rx + a[3] * ry;
    }
    v[m] = make_double2(w.x + c * ax - s * ay, w.y + s * ax + c * ay);
}

// Set-up, once per device, with that device current: look up the device address
// of the scratch array (noalloc_prepare runs it from fbim_setup).
fbim_status scratch_on_device(fbim_handle h, double2** out) {
    int dev = h->device;
    if (dev < 0 || dev >= FBIM_NOALLOC_MAX_DEVICES) {
        h->fail("fbim_apply_real_noalloc: device ordinal out of range");
        return FBIM_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(g_scratch_lock);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            h->fail(std::string("fbim_apply_real_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
            return FBIM_ERR_CUDA;
        }
        g_scratch_addr[dev] = (double2*)p;
    }
    *out = g_scratch_addr[dev];
    return FBIM_OK;
}

}  // namespace

namespace fbim {

// Run by fbim_setup with the handle's device current (see the file header): the
// scratch address, then one launch of each kernel on an empty range (N = 0: every
// thread returns before touching memory), which loads the kernels and sizes their
// local memory.
fbim_status noalloc_prepare(fbim_handle_s* h) {
    double2* scratch = nullptr;
    FBIM_TRY(scratch_on_device(h, &scratch));
    k_na_gather<<<1, 32, 0, h->stream>>>(0, h->perm, scratch, scratch);
    k_na_pairs<<<1, 32, 0, h->stream>>>(0, h->n_box, h->r_c, h->r_c * h->r_c, h->xi * h->xi, 0.0, h->cheb64,
                                        h->perm, h->cell, h->cell_start, scratch, scratch, scratch, h->flags);
    k_na_finish<<<1, 32, 0, h->stream>>>(0, h->n_p, h->band, h->slot, scratch, h->rot, h->band_dev, scratch,
                                         scratch);
    h->launches += 3;
    FBIM_CUDA_TRY(h, cudaGetLastError());
    return FBIM_OK;
}

}  // namespace fbim

extern "C" fbim_status fbim_apply_real_noalloc(fbim_handle h, const double* mu_dev, double* v_dev) {
    if (!h || !mu_dev || !v_dev) return FBIM_ERR_INVALID_ARG;
    if ((((uintptr_t)mu_dev) | ((uintptr_t)v_dev)) & 15) {
        h->fail("fbim_apply_real_noalloc: mu and v must be 16-byte aligned");
        return FBIM_ERR_INVALID_ARG;
    }
    if (h->N > FBIM_NOALLOC_MAX_NODES) {
        h->fail("fbim_apply_real_noalloc: the handle has " + std::to_string(h->N) +
                " nodes; this entry point supports at most " + std::to_string(FBIM_NOALLOC_MAX_NODES));
        return FBIM_ERR_INVALID_ARG;
    }
    if (!h->e64.ready) {
        h->fail("fbim_apply_real_noalloc: the handle's FP64 layout is missing");
        return FBIM_ERR_INVALID_ARG;
    }
    FBIM_CUDA_TRY(h, cudaSetDevice(h->device));
    double2* scratch = nullptr;
    fbim_status st = scratch_on_device(h, &scratch);
    if (st != FBIM_OK) return st;
    double2* mu_s = scratch;
    double2* v_s = scratch + FBIM_NOALLOC_MAX_NODES;
    const int N = h->N, tb = 256;
    k_na_gather<<<(N + tb - 1) / tb, tb, 0, h->stream>>>(N, h->perm, (const double2*)mu_dev, mu_s);
    k_na_pairs<<<(N + 127) / 128, 128, 0, h->stream>>>(N, h->n_box, h->r_c, h->r_c * h->r_c, h->xi * h->xi,
                                                        1.0 / (4.0 * M_PI * h->eta), h->cheb64, h->perm, h->cell,
                                                        h->cell_start, (const double2*)h->e64.off, mu_s, v_s,
                                                        h->flags);
    k_na_finish<<<(N + tb - 1) / tb, tb, 0, h->stream>>>(N, h->n_p, h->band, h->slot, v_s, h->rot, h->band_dev,
                                                         (const double2*)mu_dev, (double2*)v_dev);
    h->launches += 3;
    FBIM_CUDA_TRY(h, cudaGetLastError());
    return FBIM_OK;
}
