// Internal state and helpers of the FBIM library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>
#include <cublas_v2.h>

#include <cstdio>
#include <string>
#include <vector>

#include "../../include/fbim.h"

// stage ids for the operator's event timers
enum {
    FBIM_ST_GATHER = 0, FBIM_ST_SPREAD, FBIM_ST_FFT_F, FBIM_ST_SCALE, FBIM_ST_FFT_I,
    FBIM_ST_PAIRS, FBIM_ST_INTERP, FBIM_ST_FINISH, FBIM_N_STAGES
};

namespace fbim {

// ---------------------------------------------------------------------------
// Error plumbing: every internal call returns fbim_status; the message lands
// in the handle (or in a thread-local slot before a handle exists).
// ---------------------------------------------------------------------------
void set_global_error(const std::string& msg);
const char* global_error();

#define FBIM_CUDA_TRY(h, expr)                                                         \
    do {                                                                               \
        cudaError_t e__ = (expr);                                                      \
        if (e__ != cudaSuccess) {                                                      \
            (h)->fail(std::string(#expr) + ": " + cudaGetErrorString(e__));            \
            return e__ == cudaErrorMemoryAllocation ? FBIM_ERR_OOM : FBIM_ERR_CUDA;    \
        }                                                                              \
    } while (0)

#define FBIM_CUFFT_TRY(h, expr)                                                        \
    do {                                                                               \
        cufftResult r__ = (expr);                                                      \
        if (r__ != CUFFT_SUCCESS) {                                                    \
            (h)->fail(std::string(#expr) + ": cufft error " + std::to_string((int)r__)); \
            return FBIM_ERR_CUDA;                                                      \
        }                                                                              \
    } while (0)

#define FBIM_TRY(expr)                                                                 \
    do {                                                                               \
        fbim_status s__ = (expr);                                                      \
        if (s__ != FBIM_OK) return s__;                                                \
    } while (0)

// Device buffers of one precision of the Ewald operator.
template <typename T>
struct EwaldBuffers {
    void* off = nullptr;     // [N] T2: node offset from its cell's lower corner, cell-sorted
    void* mu_s = nullptr;    // [N] T2: forces in cell-sorted order (real space)
    void* v_s = nullptr;     // [N] T2: real-space velocities, cell-sorted
    int2* tbase = nullptr;   // [N] nearest grid point (ix, iy), tile-sorted
    void* tfrac = nullptr;   // [N] T2: x / h - base in [-1/2, 1/2], tile-sorted
    void* mu_t = nullptr;    // [N] T2: forces in tile-sorted order (wave space)
    void* v_t = nullptr;     // [N] T2: wave-space velocities, tile-sorted
    double2* mu_r = nullptr; // [N] forces rotated into their body's frame (body order, FP64)
    double2* v_band = nullptr; // [N] Alpert band velocities (body order, FP64)
    T* ring = nullptr;       // [n_tile^2][2][W][W] halo rings of the tile spread (W = TS + P - 1)
    T* grid = nullptr;       // [2][M][M] real grid (component-major)
    T* wtab = nullptr;       // [N][2][P] node window weights, tile-sorted (FP64 buffers only)
    float2* wtab_df = nullptr;  // the same weights as float-float pairs (FP64 buffers of FP32 handles)
    void* spec = nullptr;    // [2][M][M/2+1] complex half spectrum
    cufftHandle plan_f = 0;  // R2C / D2Z, batch 2
    cufftHandle plan_i = 0;  // C2R / Z2D, batch 2
    // real-space pair list in sliced-ELL layout (slices of 32 cell-sorted targets)
    void* pairs = nullptr;       // entries [slice_start[s] + k][32]: G tensor (xx, xy, yy) and source slot
    int* slice_start = nullptr;  // [n_slice + 1] entry offsets (in units of 32 entries)
    int* row_count = nullptr;    // [n_slice * 32] hits per target
    int* row_of = nullptr;       // [n_win * 256] row at each list position (-1 past N), then
                                 // [N] the list position of each row (rows sorted by length
                                 // within windows of 256)
    size_t pair_cap = 0;         // allocated entries (units of 32)
    long long n_pairs = 0;       // ordered pairs within r_c (without padding)
    long long n_padded = 0;      // stored entries including padding
    bool pairs_ready = false;
    unsigned long long pairs_geom = ~0ull;  // geometry version the pair list was built for
    // FP64 list of an FP32 handle, derived from its FP32 list: float-float entries
    // (PairEntryDF), with float-float copies of the cell offsets and of the forces
    bool pairs_df = false;
    float4* off_df = nullptr;    // [N] (x hi, x lo, y hi, y lo), cell-sorted
    float4* mu_df = nullptr;     // [N] forces, cell-sorted
    // Alpert band of the FP32 operator in float-float (FP32 buffers only): the band
    // [n_p][2 band + 1] as (hi of the 2x2 entries, lo of the 2x2 entries), and the
    // forces rotated into their body's frame (x hi, x lo, y hi, y lo), body order
    float4* band_df = nullptr;
    float4* mu_rdf = nullptr;
    // piecewise tables of its pair values (e1_piecewise): [K] piece centres, then
    // [2][K][kPwDeg + 1] float-float coefficients (S, then e^{-z}) as (hi, lo)
    float* pw = nullptr;
    int pw_K = 0;
    float pw_inv_w = 0.f, pw_kscale = 0.f;  // 1 / half-width, K / zmax
    int spread_variant = 1;      // 0: tile kernel (shared memory), 1: warp-per-node kernel
    int interp_variant = 1;      // the same for the interpolation
    float variant_ms[2][2] = {}; // autotuner timings [spread, interp][tile, warp]
    int P = 0;               // Gaussian support of this precision's wave space
    double eta_s = 0;        // its Gaussian shape
    bool ready = false;
};

// Chebyshev expansion of S(z) = (E1(z) + ln z)/2 - e^{-z} on [0, zmax], so that
// the real-space kernel coefficient E1(z)/2 - e^{-z} = S(z) - ln(z)/2.
constexpr int kChebMax = 48;
constexpr int kPwDeg = 8;  // degree of the piecewise pair-value polynomials (float-float list)
template <typename T>
struct ChebE1 {
    T c[kChebMax];
    T scale;   // 2 / zmax
    int deg;
};

// Float-float Stockham FFTs and Fourier scale of the FP64 residual operator of FP32
// handles (wave_fft.cu).
constexpr int kFftMaxPasses = 24;
struct FftPlan {
    int M = 0, nr = 0;
    int radix[kFftMaxPasses] = {};  // Stockham passes: radix 4s, then 2, 3s, 5s
};
struct WaveFft {
    int state = 0;          // 0 not set up, 1 in use, -1 unavailable (M odd, not 5-smooth or
                            // too large for shared memory)
    FftPlan plan;
    float4* tw = nullptr;   // [M] e^{-2 pi i m/M} (re hi, re lo, im hi, im lo)
    float4* tab = nullptr;  // [M/2][M][2] scale factors of the pairs (k, -k)
    float4* T1 = nullptr;   // [M][M] after the x pass, [k_x][y]
    float4* T2 = nullptr;   // [M][M] after the y pass and scale, [k_x][y]
};

}  // namespace fbim

struct fbim_handle_s {
    // ---- parameters -------------------------------------------------------
    int n_b = 0, n_p = 0, N = 0;
    double L = 0, xi = 0, r_c = 0, tol = 0, eta = 1;
    int n_box = 0, M = 0, P = 0;
    double eta_s = 0, h = 0;
    int P32 = 0;           // Gaussian support of the FP32 operator (<= P; P for FP64 handles)
    double eta_s32 = 0;    // its Gaussian shape
    int order = 4, aj = 0, aa = 0, band = 0;  // Alpert: nodes per side, window, half band
    int precision = FBIM_FP64;
    int device = 0;
    int restart = 60;
    cudaStream_t stream = nullptr;
    // the real-space pairs run on aux, forked from and joined to stream by events, so
    // that they overlap the wave-space chain (also inside captured graphs)
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    std::string err;

    // ---- geometry (device) -------------------------------------------------
    double* ref = nullptr;       // [n_p][2]
    double* Q = nullptr;         // [n_b][3]
    double* x = nullptr;         // [N][2] node positions wrapped into [0, L)
    int* cell = nullptr;         // [N] cell id of each node (body order)
    int* cell_start = nullptr;   // [n_cell + 1]
    int* cell_fill = nullptr;    // [n_cell]
    int* perm = nullptr;         // [N] slot -> node
    int* slot = nullptr;         // [N] node -> slot
    int* flags = nullptr;        // [4] device flags: 0 non-finite coordinates, 1 coincident nodes,
                                 // 3 scratch of update_positions_if_moved
    double* band_dev = nullptr;  // [n_p][2 band + 1][2][2] symmetrised M(a)_ref
    int2* gbase = nullptr;       // [N] nearest grid point of each node (body order)
    int* tile_start = nullptr;   // [n_tile^2 + 1] wave-space tiles of TS x TS grid points
    int* tile_fill = nullptr;    // [n_tile^2]
    int* tperm = nullptr;        // [N] tile slot -> node
    int* tslot = nullptr;        // [N] node -> tile slot
    int* tile_tmp = nullptr;     // [N] tile id of each node (scratch of the sort)
    int TS = 0, n_tile = 0;      // tile side (divides M) and tiles per side
    int autotune = 1;            // time the wave-space kernel variants at setup
    int tensor_cores = 1;        // FP32 block operators (preconditioner, Lanczos G) on tcgen05
    int M_min = 0;               // the grid rule's smallest side
    double grid_tune_ms = 0;     // cost of the tuned FFT pair (0: not tuned)
    int split_candidates = 0;    // cutoffs timed by the split tuner (0: not tuned)
    double split_cost_ms = 0;    // the chosen cutoff's cost per solve-equivalent
    double zmax = 0;             // xi^2 r_c^2 (upper end of the E1 expansion)
    fbim::ChebE1<double> cheb64{};
    fbim::ChebE1<float> cheb32{};

    fbim::EwaldBuffers<double> e64;
    fbim::WaveFft fft64;  // float-float transforms of the FP64 operator (FP32 handles)
    fbim::EwaldBuffers<float> e32;

    std::vector<double> host_ref;
    std::vector<double> host_band;   // symmetrised M(a)_ref band (host copy)
    double* rot = nullptr;           // [n_b][2] (cos theta, sin theta) of each body
    struct Solver* solver = nullptr; // preconditioners and Krylov workspace (solver.cu)
    struct SecondKind* sk = nullptr; // second-kind reference solver (secondkind.cu), built on first use

    // ---- stage timing (fbim_set_timing) ------------------------------------
    bool timing = false;
    cudaEvent_t ev[16] = {};
    int n_ev = 0;
    int ev_stage[16] = {};
    double stage_ms[FBIM_N_STAGES] = {};
    long long stage_calls[FBIM_N_STAGES] = {};
    void mark(int stage);          // record an event closing `stage` (no-op unless timing)
    void mark_begin();             // record the opening event of a timed operator call
    void collect();                // synchronise and accumulate the recorded intervals

    // residual audit (fbim_set_residual_audit): every mobility solve also measures its true
    // FP64 residual; the last kAuditKeep (reported, measured) pairs are kept, oldest first
    static constexpr int kAuditKeep = 64;
    bool audit = false;
    std::vector<double> audit_reported, audit_measured;

    long long launches = 0;      // kernels this library has launched on the handle (counted at launch sites)
    unsigned long long layout_version = 0;  // bumped when a buffer that launches take by pointer is reallocated
    unsigned long long geom_version = 0;    // bumped by every geometry rebuild
    struct Coarse* coarse = nullptr;        // learned coarse level (coarse.cu), NULL when off
    // the stagnation guard of GMRES suspends the coarse level for the geometry it
    // stagnated on (block-diagonal preconditioner until the next move)
    unsigned long long coarse_suspended_geom = ~0ull;
    int coarse_fallbacks = 0;

    int n_cell() const { return n_box * n_box; }
    void fail(const std::string& m) { err = m; }
};

namespace fbim {

// host setup pieces (setup_host.cu)
double host_e1(double z);
fbim_status alpert_rule(int order, std::vector<double>& v, std::vector<double>& w, int& a, std::string& err);
fbim_status alpert_reference_band(fbim_handle_s* h, std::vector<double>& band_out);
void e1_chebyshev(double zmax, int deg, std::vector<double>& coef);
// Piecewise polynomials on K equal pieces of [0, zmax] for the float-float pair values:
// on piece k, z = zc[k] + t / inv_w (zc[k] and inv_w floats, |t| <= 1.05), and
// S(z) = (E1(z) + ln z)/2 - e^{-z} = sum_j cS[k (D+1) + j] t^j (interpolated at the
// piece's Chebyshev points), e^{-z} = sum_j cE[k (D+1) + j] t^j (its Taylor series).
void e1_piecewise(double zmax, int K, int D, std::vector<float>& zc, float& inv_w, std::vector<double>& cS,
                  std::vector<double>& cE);
void g_real_host(double rx, double ry, double xi, double eta, double G[4]);
void reference_blocks(fbim_handle_s* h, const std::vector<double>& band_sym, std::vector<double>& Mr,
                      std::vector<double>& Mfull);
fbim_status choose_ewald(double L, double r_c, double tol, double xi_in, int& n_box, double& r_c_out,
                         double& xi, int& M, int& P, double& eta_s, std::string& err);
// grid autotuner (tune.cu): cheapest admissible FFT side in [M_min, 1.3 M_min]
fbim_status tune_grid(fbim_handle_s* h, int M_min, int P, int& M_out, double& best_ms);

// geometry (geometry.cu)
fbim_status build_geometry(fbim_handle_s* h);
// exclusive scan of n ints into out[0..n] (out[n] = total); out needs scan_storage(n) ints
void scan_exclusive(cudaStream_t st, const int* in, int n, int* out);
size_t scan_storage(int n);
// copy body coordinates Q_dev (device, [n_b][3]) into the handle and rebuild the geometry
fbim_status update_positions(fbim_handle_s* h, const double* Q_dev);
// The same, skipped when Q_dev holds the current body coordinates bit for bit (one
// comparison kernel and a host sync instead of the rebuild).
fbim_status update_positions_if_moved(fbim_handle_s* h, const double* Q_dev);

// solvers (solver.cu)
void free_solver(fbim_handle_s* h);
void free_second_kind(fbim_handle_s* h);  // secondkind.cu
fbim_status ensure_solver(fbim_handle_s* h);
// block preconditioner and saddle operator on x = [mu; U] (stream-ordered, no host sync)
fbim_status solver_precondition(fbim_handle_s* h, const double* in, double* out, bool fp32);
fbim_status solver_saddle(fbim_handle_s* h, const double* x, double* y, bool fp32);
// point every launch of the handle (kernels, cuFFT plans, cuBLAS) at stream s
void bind_stream(fbim_handle_s* h, cudaStream_t s);

// Brownian slip pieces (brownian.cu), stream-ordered, no host sync, in the handle's
// precision: out = G M(r) G^T in (the near-field Lanczos operator; uses the solver's
// w and r vectors as scratch) and out = G^+ in (Sec. 3.4, Eq. Gprecond-decomp)
fbim_status lanczos_operator(fbim_handle_s* h, const double* in, double* out);
fbim_status gplus_apply(fbim_handle_s* h, const double* in, double* out);
// out = G^+ G in, the projection onto the range of G (uses the solver's w as scratch)
fbim_status g_project(fbim_handle_s* h, const double* in, double* out);

// allocation-free real-space entry point (noalloc.cu): run by fbim_setup on the
// handle's device so that the entry point's first call loads and allocates nothing
fbim_status noalloc_prepare(fbim_handle_s* h);

// learned coarse level (coarse.cu)
void free_coarse(fbim_handle_s* h);
// true when the coarse level is on; refreshes its pair data if the geometry changed
// (host-synchronising: call it outside stream capture first)
bool coarse_active(fbim_handle_s* h, fbim_status* st);
fbim_status coarse_refresh(fbim_handle_s* h);
// body solve of the preconditioner with the coarse level: g = M_ref^+ R^T r_mu (per body,
// precision T), H = M_ref^+ K_ref, rU = residual of the force rows; writes mu and U
template <typename T>
fbim_status coarse_body_solve(fbim_handle_s* h, const T* g, const T* H, const double* rU, double* out_mu,
                              double* out_U);

// operators (ewald_ops.cu)
template <typename T> fbim_status ensure_ewald(fbim_handle_s* h);
template <typename T> fbim_status refresh_offsets(fbim_handle_s* h);
// which: bit 0 = real space (pairs + Alpert), bit 1 = wave space
template <typename T> fbim_status apply_operator(fbim_handle_s* h, const double* mu, double* v, int which);
// far-field noise (M(w))^1/2 W(w) into out [N][2]; Z = caller normals [M][M][2][2] or NULL (Philox)
template <typename T>
fbim_status apply_noise(fbim_handle_s* h, const double* Z, unsigned long long seed, unsigned counter, double* out);
void free_ewald(fbim_handle_s* h);
// wave_fft.cu: set up (state 1) or mark unavailable (state -1) once per handle; the
// three launches replace the FP64 FFTs and scale on the grid in place
fbim_status wfft_setup(fbim_handle_s* h);
void wfft_free(fbim_handle_s* h);
void wfft_forward(fbim_handle_s* h, cudaStream_t st, const double* grid);
void wfft_scale(fbim_handle_s* h, cudaStream_t st);
// df_out: the grid values as float-float pairs (float2 in each double's place)
void wfft_inverse(fbim_handle_s* h, cudaStream_t st, double* grid, bool df_out = false);

}  // namespace fbim
