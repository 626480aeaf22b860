// Internal declarations of libvofp: the context, launch helpers and shared device utilities.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/vofp.h"

#define VOFP_CUDA_TRY(ctx, expr)                                                        \
    do {                                                                                \
        cudaError_t e_ = (expr);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            (ctx)->set_error(std::string(#expr) + ": " + cudaGetErrorString(e_));       \
            return e_ == cudaErrorMemoryAllocation ? VOFP_ERR_OOM : VOFP_ERR_CUDA;      \
        }                                                                               \
    } while (0)

namespace vofp {

constexpr int kBX = 32;          // stencil tile width (x), one warp
constexpr int kBY = 8;           // stencil tile height (y)
constexpr int kRedThreads = 256; // threads of the streaming/reduction kernels
constexpr int kMaxPartials = 1 << 17;

// Scalars of one CG run, resident in device memory so that the loop needs no host round trip.
struct CgScalars {
    double rr;          // r.r of the (scaled) residual over the unknowns
    double rr0;         // r.r at the start of the current (inner) solve
    double pq_raw;      // p.t summed over all cells by the stencil kernel (the colour-compact
                        // red-black iteration leaves block partials for the update instead)
    double pq_corr;     // merge-group correction to p.Ap
    double alpha;       // step of the last completed iteration (used by the next stencil pass)
    double beta;        // direction coefficient for the next stencil pass
    double bnorm2;      // ||b_hat||^2 (unscaled)
    double rnorm2;      // last true ||b_hat - A_hat x||^2 (unscaled)
    double rtol;        // relative tolerance of the (outer) loop
    double inner_rtol;  // relative reduction of each inner solve (mixed precision)
    double scale;       // inner right-hand side scale (mixed precision)
    double inner_target;// relative reduction the current inner solve stops at
    double ref2;        // squared norm the current loop's tolerance is relative to
    long long iter;     // iterations of the current loop
    long long iter_total;
    long long max_iter;
    int status;         // vofp_status of the loop
    int done;           // 1 when the (outer) loop has finished
    int inner_done;     // 1 when the current inner loop has finished
    int outer;          // refinement steps
    int timing;         // 1 while the measurement hook runs: breakdowns are not recorded
    double rr_prev;     // r.r of the residual the last alpha was computed from
    int keep_dir;       // mixed precision: refinement keeps the inner search direction
    int dir_valid;      // the inner direction buffer holds a direction of this solve
};

// Work split of the compact red-black iteration kernel (chosen on the host): groups of gx x gy
// tiles (gx divides the tile columns along x, gy the tile rows), each group taking `per` work items
// of its columns, `pad` of them at the head of every column standing for no plane.
struct RbcSplit {
    int per, pad, gx, gy;
};

struct Dims {
    int nx, ny, nz;
    long long n;
    long long plane;     // nx*ny
};

}  // namespace vofp

struct vofp_ctx {
    vofp::Dims d{};
    cudaStream_t stream = nullptr;
    std::string err;
    std::vector<double> hdx, hdy, hdz;
    double *dx = nullptr, *dy = nullptr, *dz = nullptr;

    bool built = false;
    int bc[6] = {0, 0, 0, 0, 0, 0};
    vofp_phys phys{};
    bool dirichlet = false;
    double* nflux[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    bool has_nflux[6] = {false, false, false, false, false, false};

    // operator (FP64, unscaled): T of each cell's +face, full diagonal of the unmerged operator
    double *Tx = nullptr, *Ty = nullptr, *Tz = nullptr, *diag = nullptr;
    // effective apertures (faces of cells without an unknown closed)
    double *axe = nullptr, *aye = nullptr, *aze = nullptr;
    // symmetric scaling: s = diag(A_hat)^-1/2 of the cell's group, sq = 1/s (0 without unknown)
    double *s = nullptr, *sq = nullptr;
    double *Txs = nullptr, *Tys = nullptr, *Tzs = nullptr;     // s_L T s_R
    float *Txf = nullptr, *Tyf = nullptr, *Tzf = nullptr;      // FP32 copies
    uint32_t* slave_bits = nullptr;   // bit c set when c belongs to another cell's group
    // red-black elimination (Eisenstat form of red-black symmetric Gauss-Seidel): bit c of red_bits
    // is set for "red" cells -- (i+j+k) even, with an unknown, in no merge group -- whose unknowns
    // are eliminated; excl_bits = slave_bits | red_bits marks cells left out of the reduced dots
    double* rho = nullptr;            // cell density (after the optional smoothing)
    // inverse face resistance 1/((d_L rho_L + d_R rho_R)/2) of each cell's open +x, +y, +z face
    double *kx = nullptr, *ky = nullptr, *kz = nullptr;
    uint32_t* red_bits = nullptr;
    float* Tzr = nullptr;             // Tzf with the sign bit set on red cells (red flag)
    uint32_t* excl_bits = nullptr;
    long long n_red = 0;
    int32_t* root = nullptr;          // group root per cell, -1 without unknown
    uint8_t* inactive = nullptr;
    // merge groups with more than one cell: cells of group g are gcells[gptr[g] .. gptr[g+1]),
    // master first; gcorr[g] = s_m^2 * sum of the cells' diagonals - |G|
    int ngroups = 0;
    int *gptr = nullptr, *gcells = nullptr;
    double* gcorr = nullptr;
    long long gptr_cap = 0, gcells_cap = 0;   // allocated entries of gptr (and gcorr) and gcells
    // small cells of the last build, in arrival order (device; kept across builds)
    long long small_cap = 0;
    long long *small_cells = nullptr, *small_targets = nullptr;
    double* small_vf = nullptr;
    int32_t* small_tslot = nullptr;
    long long n_unknowns = 0, n_inactive = 0, n_merged = 0;

    // Krylov workspace
    double *xt = nullptr, *r = nullptr, *p0 = nullptr, *p1 = nullptr, *q = nullptr, *bt = nullptr;
    float *rf = nullptr, *pf0 = nullptr, *pf1 = nullptr, *qf = nullptr, *xf = nullptr;
    float* qf2 = nullptr;             // flexible CG (learned preconditioner): second q buffer
    char* fcg = nullptr;              // flexible CG scalars (device)
    double* partials = nullptr;       // block partial sums
    unsigned int* counters = nullptr; // last-block tickets
    vofp::CgScalars* sc = nullptr;
    double* work = nullptr;           // apply / residual scratch (cells)
    double* dstage = nullptr;         // host-call staging: b, x and one set of inputs
    double* dstage2 = nullptr;        // a second set of inputs (batched host calls)
    size_t dstage_bytes = 0;

    // CUDA graphs of the solve loops, keyed by configuration
    cudaGraphExec_t graph_fp64 = nullptr;
    int graph_fp64_key = -1;
    cudaGraphExec_t graph_mixed = nullptr;
    int graph_mixed_key = -1;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // vofp_solve_host(_batch): a copy stream that brings the face velocities in while the operator
    // builds, and the next step's inputs while a step solves
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t copy_done = nullptr;
    cudaEvent_t ops_done = nullptr;
    cudaEvent_t set_ready[2] = {nullptr, nullptr};

    size_t bytes = 0;
    std::vector<void*> allocs;
    long long launches = 0;           // kernels launched (graph bodies counted per execution)
    int pdl = 1;                      // programmatic dependent launch in the mixed inner loop
    cudaError_t launch_err = cudaSuccess;  // first failed extended launch since it was cleared
    bool kernels_prepared = false;    // dynamic shared memory opted in, occupancies queried
    // TMA-fed CG stencil: usable per precision (row pitch a multiple of 16 bytes, driver entry
    // point found, not disabled by VOFP_STENCIL_TMA=0); resident blocks per SM; encoded maps
    bool tma_ok[2] = {false, false};  // FP32, FP64
    int tma_blocks_per_sm[2] = {0, 0};
    int tma_cpt32 = 2;                // FP32 TMA stencil: cells per thread along x
    bool rb_tma_ok = false;           // FP32 red-black iteration fed by bulk tensor copies
    // colour-compact FP32 vectors of the red-black inner solve (vofp_rbc.cu): black cell of each x
    // pair (N/2), then the even-parity merge-group cells ("exceptions"); built per operator
    bool rbc_ok = false;              // usable for the current operator
    bool rbc_built = false;           // structures built for the current operator
    long long rbc_nh = 0;             // N/2
    int rbc_ne = 0, rbc_nf = 0;       // exceptions, rows next to an exception
    float *rbc_r = nullptr, *rbc_p0 = nullptr, *rbc_p1 = nullptr, *rbc_x = nullptr, *rbc_q = nullptr;
    uint32_t* rbc_bits = nullptr;     // compact entries excluded from the dots (copies of a group value)
    int* rbc_exc = nullptr;           // exception cells
    int *rbc_fcell = nullptr, *rbc_fexc = nullptr;   // rows next to exceptions, exception per face
    int* rbc_fh = nullptr;            // compact index per fix row (-1: a merge-group member)
    float* rbc_fT = nullptr;          // face coefficient per fix row and face (0: no exception)
    int* rbc_enb = nullptr;           // per exception and face: the compact index of the black pair
    float* rbc_eT = nullptr;          // per exception and face: the coefficient (0 at the boundary)
    float* rbc_dE = nullptr;          // per exception: red formula - p (entry ne: 0)
    int *rbc_gref = nullptr, *rbc_gfx = nullptr;     // compact / fix-row index of every gcells entry
    int *rbc_gm = nullptr, *rbc_gf = nullptr;        // per group: four members' compact / fix-row index
    int* rbc_gn = nullptr;            // per group: member count
    // VOF operator (vofp_vof.cu): corrected stage velocities, two stage buffers, interface planes
    double *vof_uxh = nullptr, *vof_uyh = nullptr, *vof_wmh = nullptr, *vof_wph = nullptr;
    double *vof_phi = nullptr, *vof_plic = nullptr;
    double* rk2_buf = nullptr;        // RK2 step (vofp_rk2.cu): face fields and cell arrays
    long long rbc_cap = 0;            // allocated compact length
    int rbc_blocks_per_sm = 0;
    int rbc_rpt = 2;                  // rows per thread of the compact iteration kernel (tile 32 x 8 rpt)
    int rbc_nblocks = 0;              // iteration kernel blocks and work split (see rbc_split)
    vofp::RbcSplit rbc_split{};
    int tma_blocks_deep32 = 0;        // resident blocks per SM of the six-stage FP32 stencil
    int rb_tma_blocks_per_sm = 0;
    std::map<std::tuple<const void*, int, int>, CUtensorMap> tma_maps;

    void set_error(const std::string& m) { err = m; }
    template <typename T>
    vofp_status alloc(T** p, size_t count) {
        void* q = nullptr;
        cudaError_t e = cudaMalloc(&q, sizeof(T) * (count ? count : 1));
        if (e != cudaSuccess) {
            set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
            return VOFP_ERR_OOM;
        }
        allocs.push_back(q);
        bytes += sizeof(T) * count;
        *p = reinterpret_cast<T*>(q);
        return VOFP_OK;
    }
};

namespace vofp {

// ---- launches implemented in the .cu files -------------------------------------------------
// TMA-fed CG stencil (vofp_tma.cu): per-context preparation, and one launch when the context's
// tensor maps can be built (returns false otherwise; the caller then uses the register kernel)
void prepare_tma(vofp_ctx* c);
// cached 3-D tensor map of an FP32 nx x ny x nz array with a bw x bh x 1 box (null if it cannot be built)
const CUtensorMap* tensor_map_f32(vofp_ctx* c, const float* ptr, int bw, int bh);
// the same for an nxe x ny x nz array (the colour-compact vectors: nxe = nx/2)
const CUtensorMap* tensor_map_f32_x(vofp_ctx* c, const float* ptr, int nxe, int bw, int bh);
// TMA-fed fused red-black iteration, FP32 (vofp_rb_tma.cu): preparation and one launch (false
// when it cannot run on this context; the caller then uses the register-prefetch kernel)
void prepare_rb_tma(vofp_ctx* c);
bool launch_cg_rb_tma(vofp_ctx* c, cudaStream_t st, const float* r, const float* po, float* pn, float* xv, float* q);
// colour-compact red-black inner solve (vofp_rbc.cu)
vofp_status rbc_ensure(vofp_ctx* c);   // build the compact structures if eligible; sets c->rbc_ok
void rbc_prep(vofp_ctx* c, cudaStream_t st, const double* rhs);   // inner start from the FP64 reduced rhs
void rbc_iteration(vofp_ctx* c, cudaStream_t st, const float* po, float* pn, cudaGraphConditionalHandle h,
                   int use_h);
void rbc_finish_xf(vofp_ctx* c, cudaStream_t st);                 // xf (full grid) = x_c + alpha p0_c
void rbc_time_kernel(vofp_ctx* c, cudaStream_t st);               // one iteration kernel launch
void rbc_time_aux(vofp_ctx* c, cudaStream_t st);                  // the exception and group kernels of one iteration
template <typename V>
bool launch_cg_tma(vofp_ctx* c, cudaStream_t st, const V* Tx, const V* Ty, const V* Tz, const V* r, const V* po,
                   V* pn, V* xv, V* q);

vofp_status build_operator(vofp_ctx* c, const double* F, const double* ax, const double* ay,
                           const double* az, const double* vf, const vofp_bc* bc,
                           const vofp_phys* phys);
vofp_status rhs(vofp_ctx* c, const double* u, const double* v, const double* w,
                const double* body, double* b);
vofp_status apply_unscaled(vofp_ctx* c, const double* x, double* y);
vofp_status residual(vofp_ctx* c, const double* b, const double* x, double* rel);
vofp_status solve(vofp_ctx* c, const double* b, double* x, const vofp_solve_opts* o,
                  vofp_solve_info* info);
vofp_status solve_fcg(vofp_ctx* c, const double* b, double* x, const vofp_solve_opts* o, vofp_solve_info* info);
vofp_status scaled_pair(vofp_ctx* c, const double* b, const double* x, float* r_scaled, float* x_scaled);
vofp_status nn_train_anorm(vofp_ctx* c, vofp_nn* nn, const float* r, const float* e, float lr, int update,
                           float* loss);
vofp_status time_iteration_kernels(vofp_ctx* c, int precision, bool rb, int reps, float* st, float* up,
                                   float* red);

// group helpers (vofp_assemble.cu)
// Scalars at the start of an inner (FP32) solve, set by the block that completes the reduction of
// the new inner residual: t = r_f . r_f of the normalised residual, rr = ||r||^2 before
// normalisation.  With the direction kept (reliable update), beta rescales the old direction.
__device__ inline void inner_start_scalars(CgScalars* sc, double t, double rr, bool keep) {
    const double scale_old = sc->scale;
    const double scale_new = (rr > 0.0 && !sc->done) ? sqrt(rr) : 0.0;
    sc->scale = scale_new;
    // the last refinement step only needs the reduction that reaches rtol (with margin)
    const double need = sc->rnorm2 > 0.0 ? 0.3 * sc->rtol * sqrt(sc->ref2 / sc->rnorm2) : 1.0;
    sc->inner_target = fmax(sc->inner_rtol, fmin(need, 0.5));
    double beta = 0.0;
    if (keep && scale_old > 0.0 && sc->rr_prev > 0.0) {
        beta = scale_new / (scale_old * sc->rr_prev);
        if (!isfinite(beta)) beta = 0.0;
    }
    sc->rr = t;
    sc->alpha = 0.0;
    sc->beta = beta;
    sc->iter = 0;
    sc->inner_done = 0;
    sc->rr0 = t;
    sc->dir_valid = sc->keep_dir;
}

// face and cell indexing: x faces (nx+1) x ny x nz, y faces nx x (ny+1) x nz, z faces nx x ny x (nz+1)
__device__ __forceinline__ long long fx_idx(const Dims& d, int i, int j, int k) {
    return i + (long long)(d.nx + 1) * (j + (long long)d.ny * k);
}
__device__ __forceinline__ long long fy_idx(const Dims& d, int i, int j, int k) {
    return i + (long long)d.nx * (j + (long long)(d.ny + 1) * k);
}
__device__ __forceinline__ long long fz_idx(const Dims& d, int i, int j, int k) {
    return i + (long long)d.nx * (j + (long long)d.ny * k);
}
// cell counts stay below 2^31 (checked by vofp_create): 32-bit division is enough
__device__ __forceinline__ void cell_ijk(const Dims& d, long long c, int& i, int& j, int& k) {
    const unsigned int uc = (unsigned int)c, nx = (unsigned int)d.nx, ny = (unsigned int)d.ny;
    const unsigned int t = uc / nx;
    i = int(uc - t * nx);
    const unsigned int kk = t / ny;
    j = int(t - kk * ny);
    k = int(kk);
}

// projection of the face velocities and its divergence check (vofp_project.cu)
vofp_status project(vofp_ctx* c, const double* p, const double* u, const double* v, const double* w,
                    const double* body, double* uo, double* vo, double* wo, double* div, double* max_div);

// VOF operator of Sec. 2.4 (vofp_vof.cu)
vofp_status vof_flux_correct(vofp_ctx* c, const double* ax, const double* ay, const double* az, const double* u,
                             const double* v, const double* w, double* uxh, double* uyh, double* wmh, double* wph);
vofp_status vof_advect(vofp_ctx* c, const double* F, const double* ax, const double* ay, const double* az,
                       const double* vf, const double* u, const double* v, const double* w, double dt, int order,
                       double* F_out);

// exit flux of the radiation condition, installed as the +x face's prescribed flux (vofp_exit.cu)
vofp_status exit_flux(vofp_ctx* c, const double* u, const double* v, const double* w, const double* body, double uc,
                      const double* r1, int balance, double* g_out, double* shift_out);

void launch_group_expand(vofp_ctx* c, double* v);
void launch_group_fold(vofp_ctx* c, double* v, bool zero_slaves);

// stencil helpers (vofp_stencil.cu)
// t = A x on the full grid with the unscaled coefficients and explicit diagonal
void launch_stencil_apply_unscaled(vofp_ctx* c, const double* x, double* t);
// t = (unit-diagonal scaled operator) x, FP64
void launch_stencil_apply_scaled(vofp_ctx* c, const double* x, double* t);
// merge-group patch after a scaled stencil: q_m = sum t + corr p_m, expanded; p.Ap correction
template <typename V>
void launch_group_patch(vofp_ctx* c, V* t, const V* p, bool dot_correction);

// Launch a kernel on stream s and count it.
template <typename... KArgs, typename... Args>
inline void launch(vofp_ctx* c, void (*k)(KArgs...), dim3 g, dim3 b, cudaStream_t s, Args... args) {
    k<<<g, b, 0, s>>>(static_cast<KArgs>(args)...);
    ++c->launches;
}
// Same, with dynamic shared memory.
template <typename... KArgs, typename... Args>
inline void launch_smem(vofp_ctx* c, void (*k)(KArgs...), dim3 g, dim3 b, size_t smem, cudaStream_t s,
                        Args... args) {
    k<<<g, b, smem, s>>>(static_cast<KArgs>(args)...);
    ++c->launches;
}

// Same, optionally as a programmatic dependent launch: the kernel may be scheduled while the
// previous kernel on the stream drains, and must call griddepcontrol.wait before it reads what
// that kernel wrote. A refused launch is recorded in c->launch_err.
template <typename... KArgs, typename... Args>
inline void launch_dep(vofp_ctx* c, bool pdl, void (*k)(KArgs...), dim3 g, dim3 b, size_t smem, cudaStream_t s,
                       Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = g;
    cfg.blockDim = b;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
    if (e != cudaSuccess && c->launch_err == cudaSuccess) c->launch_err = e;
    ++c->launches;
}

namespace nn {
long long bound_cells(const vofp_nn* n);
cudaStream_t stream_of(const vofp_nn* n);
// one forward pass of the bound network on stream st (r: scaled residual, FP32 cells); the result
// stays in the network's output buffer, output(n)
vofp_status forward_on(vofp_nn* n, cudaStream_t st, const float* r);
float* output(vofp_nn* n);
int forward_kernels(const vofp_nn* n);           // kernels one forward pass launches
vofp_status read_device_error(vofp_nn* n);       // VOFP_ERR_DEVICE_TIMEOUT if a bounded wait ran out
vofp_status prepare_training(vofp_nn* n);        // gradient buffers
// after forward_on: gradients from a given dL/dz of the output (FP32 cells), Adam step if update
vofp_status train_from_grad_on(vofp_nn* n, cudaStream_t st, const float* dz, float lr, int update);
}  // namespace nn

inline int ceil_div(long long a, long long b) { return int((a + b - 1) / b); }

inline int num_sms() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

}  // namespace vofp

// ---- device utilities ------------------------------------------------------------------------
namespace vofp {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum of v over the block, valid in thread 0.  Fixed order: deterministic.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int w = 0; w < NT / 32; ++w) s += sh[w];
    }
    return s;
}

// Write this block's partial and, in the block that finishes last, reduce all partials in
// index order.  Returns true (in thread 0 of the last block) with *total set.
// The ticket counter is reset by the last block for the next launch.
__device__ __forceinline__ bool last_block_reduce(double part, double* partials,
                                                  unsigned int* counter, int nblocks,
                                                  double* total, double* sh) {
    __shared__ bool is_last;
    const int b = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    if (threadIdx.x + blockDim.x * threadIdx.y == 0) {
        partials[b] = part;
        __threadfence();
        unsigned int t = atomicAdd(counter, 1u);
        is_last = (t == (unsigned int)(nblocks - 1));
    }
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int nt = blockDim.x * blockDim.y;
    double s = 0.0;
    if (tid < 32) {
        for (int i = tid; i < nblocks; i += 32) s += *((volatile double*)&partials[i]);
        s = warp_sum(s);
    }
    if (tid == 0) {
        *total = s;
        *counter = 0u;
    }
    (void)nt;
    (void)sh;
    return tid == 0;
}

}  // namespace vofp
