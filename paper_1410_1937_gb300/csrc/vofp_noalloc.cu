// Residual norm ||b_hat - A_hat x|| / ||b_hat|| that allocates no device memory.
//
// vofp_residual computes the same number with per-cell scratch vectors of the context and may
// allocate the solver workspace on its first use.  Callers that must not allocate once set-up is
// over -- a time-step loop whose device memory is owned by another allocator (a framework's
// caching pool that keeps all free memory, where a direct cudaMalloc fails or forces the pool to
// release memory), a process with a fixed memory budget, or code that cannot accept the implicit
// device synchronisation of cudaMalloc/cudaFree -- use vofp_residual_noalloc instead.  Its only
// scratch is the file-scope array below, sized for at most kNaMaxGroups merge groups; every GPU
// that loads the library holds it until the process exits.
//
// The cell pass evaluates the 7-point operator on the fly, reading x at each neighbour's group
// master, so no expanded copy of x is stored.  A cell whose neighbour has it as root is the master
// of a merge group (every group's master touches one of its members); its row is summed by the
// group pass instead.  All sums are block partials reduced in index order: the result is
// deterministic.
#include <cmath>
#include <mutex>
#include <string>

#include "vofp_internal.cuh"

namespace {

constexpr int kNaThreads = 256;
constexpr int kNaBlocks = 1024;          // block partials per pass
constexpr int kNaMaxGroups = 1 << 16;    // merge groups whose sums the scratch holds
// layout (doubles): group r_hat [kNaMaxGroups] | group b_hat [kNaMaxGroups] |
//                   cell partials 2 x kNaBlocks | result 2.
// Every slot a call reads is written earlier in the same call, so nothing needs clearing; calls
// that overlap on the GPU (other streams, other threads) share the array and race.
constexpr int kOffGroupB = kNaMaxGroups;
constexpr int kOffPart = 2 * kNaMaxGroups;
constexpr int kOffResult = kOffPart + 2 * kNaBlocks;
constexpr int kScratchDoubles = kOffResult + 2;   // about 1.03 MB

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

std::mutex g_mu;
double* g_addr[64] = {};   // device address of the array, per device ordinal

__device__ __forceinline__ double warp_sum_na(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double block_sum_na(double v, double* sh) {
    v = warp_sum_na(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kNaThreads / 32; ++w) s += sh[w];
    __syncthreads();
    return s;
}

// (A x_hat)_c with the unscaled coefficients; *master is set when a neighbour has c as root
__device__ __forceinline__ double row_apply(const vofp::Dims& d, long long c, int i, int j, int k,
                                            const double* __restrict__ Tx, const double* __restrict__ Ty,
                                            const double* __restrict__ Tz, const double* __restrict__ diag,
                                            const int32_t* __restrict__ root, const double* __restrict__ x,
                                            bool* master) {
    double t = diag[c] * x[root[c]];
    bool m = false;
    auto nb = [&](long long n, double T) {
        const int32_t r = root[n];
        m |= (r == (int32_t)c) && (n != c);
        if (r >= 0) t = fma(-T, x[r], t);
    };
    if (i > 0) nb(c - 1, Tx[c - 1]);
    if (i < d.nx - 1) nb(c + 1, Tx[c]);
    if (j > 0) nb(c - d.nx, Ty[c - d.nx]);
    if (j < d.ny - 1) nb(c + d.nx, Ty[c]);
    if (k > 0) nb(c - d.plane, Tz[c - d.plane]);
    if (k < d.nz - 1) nb(c + d.plane, Tz[c]);
    *master = m;
    return t;
}

// pass 1: cells that are their own unknown and not the master of a group
__global__ void __launch_bounds__(kNaThreads)
k_na_cells(vofp::Dims d, const double* __restrict__ Tx, const double* __restrict__ Ty,
           const double* __restrict__ Tz, const double* __restrict__ diag, const int32_t* __restrict__ root,
           const double* __restrict__ b, const double* __restrict__ x, double* __restrict__ scratch) {
    __shared__ double sh[kNaThreads / 32];
    double rr = 0.0, bb = 0.0;
    const long long rows = (long long)d.ny * d.nz;
    for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
        const int j = int(row % d.ny), k = int(row / d.ny);
        for (int i = threadIdx.x; i < d.nx; i += blockDim.x) {
            const long long c = i + d.nx * row;
            if (root[c] != (int32_t)c) continue;
            bool master;
            const double t = row_apply(d, c, i, j, k, Tx, Ty, Tz, diag, root, x, &master);
            if (master) continue;
            const double r = b[c] - t;
            rr = fma(r, r, rr);
            bb = fma(b[c], b[c], bb);
        }
    }
    rr = block_sum_na(rr, sh);
    bb = block_sum_na(bb, sh);
    if (threadIdx.x == 0) {
        scratch[kOffPart + blockIdx.x] = rr;
        scratch[kOffPart + kNaBlocks + blockIdx.x] = bb;
    }
}

// pass 2: one thread per merge group sums its cells' rows and right-hand sides
__global__ void __launch_bounds__(kNaThreads)
k_na_groups(vofp::Dims d, int ng, const int* __restrict__ gptr, const int* __restrict__ gcells,
            const double* __restrict__ Tx, const double* __restrict__ Ty, const double* __restrict__ Tz,
            const double* __restrict__ diag, const int32_t* __restrict__ root, const double* __restrict__ b,
            const double* __restrict__ x, double* __restrict__ scratch) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x) {
        double r = 0.0, bh = 0.0;
        for (int u = gptr[g]; u < gptr[g + 1]; ++u) {
            const long long c = gcells[u];
            const int i = int(c % d.nx);
            const long long t2 = c / d.nx;
            const int j = int(t2 % d.ny), k = int(t2 / d.ny);
            bool m;
            r += b[c] - row_apply(d, c, i, j, k, Tx, Ty, Tz, diag, root, x, &m);
            bh += b[c];
        }
        scratch[g] = r;
        scratch[kOffGroupB + g] = bh;
    }
}

// pass 3 (one block): index-order sums of the cell partials and the group values
__global__ void __launch_bounds__(kNaThreads) k_na_final(int nblocks, int ng, double* __restrict__ scratch) {
    __shared__ double sh[kNaThreads / 32];
    double rr = 0.0, bb = 0.0;
    for (int p = threadIdx.x; p < nblocks; p += blockDim.x) {
        rr += scratch[kOffPart + p];
        bb += scratch[kOffPart + kNaBlocks + p];
    }
    for (int g = threadIdx.x; g < ng; g += blockDim.x) {
        rr = fma(scratch[g], scratch[g], rr);
        bb = fma(scratch[kOffGroupB + g], scratch[kOffGroupB + g], bb);
    }
    rr = block_sum_na(rr, sh);
    bb = block_sum_na(bb, sh);
    if (threadIdx.x == 0) {
        scratch[kOffResult] = rr;
        scratch[kOffResult + 1] = bb;
    }
}

}  // namespace

extern "C" vofp_status vofp_residual_noalloc(vofp_ctx* c, const double* b, const double* x, double* rel) {
    if (!c) return VOFP_ERR_INVALID_ARG;
    c->err.clear();
    if (!c->built) {
        c->set_error("vofp_build_operator has not succeeded on this context");
        return VOFP_ERR_NOT_BUILT;
    }
    if (!b || !x || !rel) {
        c->set_error("null input");
        return VOFP_ERR_INVALID_ARG;
    }
    if (c->ngroups > kNaMaxGroups) {
        c->set_error("vofp_residual_noalloc: the operator has " + std::to_string(c->ngroups) +
                     " merge groups; the fixed scratch holds at most " + std::to_string(kNaMaxGroups));
        return VOFP_ERR_INVALID_ARG;
    }
    int dev = 0;
    VOFP_CUDA_TRY(c, cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        c->set_error("device ordinal out of range");
        return VOFP_ERR_INVALID_ARG;
    }
    double* scratch = nullptr;
    {
        // once per device, with that device current: the array's device address
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_addr[dev]) {
            void* p = nullptr;
            VOFP_CUDA_TRY(c, cudaGetSymbolAddress(&p, g_noalloc_scratch));
            g_addr[dev] = static_cast<double*>(p);
        }
        scratch = g_addr[dev];
    }
    const vofp::Dims d = c->d;
    cudaStream_t st = c->stream;
    const long long rows = (long long)d.ny * d.nz;
    const int nb = (int)(rows < kNaBlocks ? rows : kNaBlocks);
    k_na_cells<<<nb, kNaThreads, 0, st>>>(d, c->Tx, c->Ty, c->Tz, c->diag, c->root, b, x, scratch);
    ++c->launches;
    if (c->ngroups > 0) {
        k_na_groups<<<vofp::ceil_div(c->ngroups, kNaThreads), kNaThreads, 0, st>>>(
            d, c->ngroups, c->gptr, c->gcells, c->Tx, c->Ty, c->Tz, c->diag, c->root, b, x, scratch);
        ++c->launches;
    }
    k_na_final<<<1, kNaThreads, 0, st>>>(nb, c->ngroups, scratch);
    ++c->launches;
    VOFP_CUDA_TRY(c, cudaGetLastError());
    double h[2];
    VOFP_CUDA_TRY(c, cudaMemcpyAsync(h, scratch + kOffResult, sizeof(h), cudaMemcpyDeviceToHost, st));
    VOFP_CUDA_TRY(c, cudaStreamSynchronize(st));
    *rel = h[1] > 0.0 ? std::sqrt(h[0] / h[1]) : std::sqrt(h[0]);
    return VOFP_OK;
}
