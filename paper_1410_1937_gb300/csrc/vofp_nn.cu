// Learned preconditioner: a 3-level 3-D convolutional encoder-decoder (16/32/64 channels, 3x3x3
// kernels, zero padding, ReLU, 2x2x2 average pooling, nearest upsampling, skip concatenation, a
// final 1x1x1 layer) that maps the operator's geometry and a residual to an approximate solution
// of the scaled pressure system.  The paper has no counterpart: the network is used as the
// preconditioner and initial guess of a flexible CG around the paper's conjugate-gradient solve.
//
// Activations are BF16 in channels-last layout ((z*ny + y)*nx + x)*C + c; weights are kept as FP32
// masters (Adam) with BF16 copies; every 3x3x3 convolution is an implicit GEMM on the tensor cores
// (mma.sync m16n8k16, BF16 inputs, FP32 accumulation): M = 16 output voxels along x per warp,
// N = output channels, K = 27 taps x input channels.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <random>
#include <vector>

#include "vofp_internal.cuh"

namespace vofp {
namespace nn {

using bf16 = __nv_bfloat16;

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t ld32(const bf16* p) { return *reinterpret_cast<const uint32_t*>(p); }
__device__ __forceinline__ uint32_t pack2(bf16 lo, bf16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// ---- 3x3x3 convolution, forward (also the data gradient, with flipped/transposed weights) ----
// in: (nx,ny,nz,cin) BF16, cin % 16 == 0; w: [27][COUT][cin] BF16; out: (nx,ny,nz,COUT) BF16.
// bias may be null; relu applies max(0, .).  A warp owns 16 consecutive voxels of one x-row.
template <int COUT>
__global__ void __launch_bounds__(128)
k_conv3(const bf16* __restrict__ in, int cin, const bf16* __restrict__ w, const float* __restrict__ bias,
        bf16* __restrict__ out, int nx, int ny, int nz, int relu) {
    constexpr int NT = COUT / 8;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int x0 = (blockIdx.x * 4 + warp) * 16;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x0 >= nx) return;
    float acc[NT][4];
#pragma unroll
    for (int n = 0; n < NT; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
    const int xa = x0 + g, xb = x0 + g + 8;
    for (int tap = 0; tap < 27; ++tap) {
        const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
        const int iz = z + dz, iy = y + dy;
        if (iz < 0 || iz >= nz || iy < 0 || iy >= ny) continue;
        const int ixa = xa + dx, ixb = xb + dx;
        const bool va = ixa >= 0 && ixa < nx && xa < nx, vb = ixb >= 0 && ixb < nx && xb < nx;
        const long long rowbase = ((long long)iz * ny + iy) * nx;
        const bf16* pa = in + (rowbase + ixa) * cin;
        const bf16* pb = in + (rowbase + ixb) * cin;
        const bf16* wt = w + (long long)tap * COUT * cin;
        for (int kc = 0; kc < cin; kc += 16) {
            uint32_t a[4];
            a[0] = va ? ld32(pa + kc + 2 * t) : 0u;
            a[1] = vb ? ld32(pb + kc + 2 * t) : 0u;
            a[2] = va ? ld32(pa + kc + 2 * t + 8) : 0u;
            a[3] = vb ? ld32(pb + kc + 2 * t + 8) : 0u;
#pragma unroll
            for (int n = 0; n < NT; ++n) {
                const bf16* pw = wt + (long long)(n * 8 + g) * cin + kc + 2 * t;
                mma16816(acc[n], a, ld32(pw), ld32(pw + 8));
            }
        }
    }
    const long long ob = ((long long)z * ny + y) * nx;
#pragma unroll
    for (int n = 0; n < NT; ++n) {
        const int co = n * 8 + 2 * t;
        float b0 = bias ? bias[co] : 0.f, b1 = bias ? bias[co + 1] : 0.f;
        float v0 = acc[n][0] + b0, v1 = acc[n][1] + b1, v2 = acc[n][2] + b0, v3 = acc[n][3] + b1;
        if (relu) {
            v0 = fmaxf(v0, 0.f); v1 = fmaxf(v1, 0.f); v2 = fmaxf(v2, 0.f); v3 = fmaxf(v3, 0.f);
        }
        if (xa < nx) *reinterpret_cast<__nv_bfloat162*>(out + (ob + xa) * COUT + co) = __floats2bfloat162_rn(v0, v1);
        if (xb < nx) *reinterpret_cast<__nv_bfloat162*>(out + (ob + xb) * COUT + co) = __floats2bfloat162_rn(v2, v3);
    }
}

// ---- 3x3x3 convolution, weight gradient ---------------------------------------------------
// dw[tap][co][ci] += sum over voxels v of dy[v][co] * x[v + tap - 1][ci] (FP32 atomics into dw).
// GEMM per tap: M = 16 output channels (co tile), N = input channels, K = 16 voxels of an x-row.
template <int CIN>
__global__ void __launch_bounds__(128)
k_conv3_wgrad(const bf16* __restrict__ x, const bf16* __restrict__ dy, int cout, float* __restrict__ dw,
              int nx, int ny, int nz, int rows_per_block) {
    constexpr int NT = CIN / 8;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int cotiles = cout / 16;
    const int tap = blockIdx.x / cotiles, co0 = (blockIdx.x % cotiles) * 16;
    const int dz = tap / 9 - 1, dy_ = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
    float acc[NT][4];
#pragma unroll
    for (int n = 0; n < NT; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
    const long long rows = (long long)ny * nz;
    const long long r0 = (long long)blockIdx.y * rows_per_block;
    const long long r1 = min(rows, r0 + rows_per_block);
    const bf16 zero = __float2bfloat16(0.f);
    for (long long row = r0; row < r1; ++row) {
        const int y = int(row % ny), z = int(row / ny);
        const int iy = y + dy_, iz = z + dz;
        const bool rowok = iy >= 0 && iy < ny && iz >= 0 && iz < nz;
        const long long ob = row * nx, ib = ((long long)iz * ny + iy) * nx;
        for (int xs = warp * 16; xs < nx; xs += 64) {
            // K index k = voxel xs + k of this row
            auto dyv = [&](int k, int m) -> bf16 {
                const int xx = xs + k;
                return xx < nx ? dy[(ob + xx) * cout + co0 + m] : zero;
            };
            auto xv = [&](int k, int ci) -> bf16 {
                const int xx = xs + k, ix = xx + dx;
                return (rowok && xx < nx && ix >= 0 && ix < nx) ? x[(ib + ix) * CIN + ci] : zero;
            };
            uint32_t a[4];
            a[0] = pack2(dyv(2 * t, g), dyv(2 * t + 1, g));
            a[1] = pack2(dyv(2 * t, g + 8), dyv(2 * t + 1, g + 8));
            a[2] = pack2(dyv(2 * t + 8, g), dyv(2 * t + 9, g));
            a[3] = pack2(dyv(2 * t + 8, g + 8), dyv(2 * t + 9, g + 8));
#pragma unroll
            for (int n = 0; n < NT; ++n) {
                const int ci = n * 8 + g;
                const uint32_t b0 = pack2(xv(2 * t, ci), xv(2 * t + 1, ci));
                const uint32_t b1 = pack2(xv(2 * t + 8, ci), xv(2 * t + 9, ci));
                mma16816(acc[n], a, b0, b1);
            }
        }
    }
    // c0,c1: (co0 + g, ci = n*8 + 2t, +1); c2,c3: (co0 + g + 8, same ci)
    float* base = dw + (long long)tap * cout * CIN;
#pragma unroll
    for (int n = 0; n < NT; ++n) {
        const int ci = n * 8 + 2 * t;
        atomicAdd(base + (long long)(co0 + g) * CIN + ci, acc[n][0]);
        atomicAdd(base + (long long)(co0 + g) * CIN + ci + 1, acc[n][1]);
        atomicAdd(base + (long long)(co0 + g + 8) * CIN + ci, acc[n][2]);
        atomicAdd(base + (long long)(co0 + g + 8) * CIN + ci + 1, acc[n][3]);
    }
}

// ---- small kernels --------------------------------------------------------------------------
// BF16 weights: wb[tap][co][ci] from FP32 masters; the data-gradient copy wt[26-tap][ci][co]
__global__ void k_weights_bf16(const float* __restrict__ w, bf16* __restrict__ wb, bf16* __restrict__ wt,
                               int cout, int cin) {
    const int n = 27 * cout * cin;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int ci = i % cin, co = (i / cin) % cout, tap = i / (cin * cout);
        const bf16 v = __float2bfloat16(w[i]);
        wb[i] = v;
        if (wt) wt[((long long)(26 - tap) * cin + ci) * cout + co] = v;
    }
}

// dpre = dy where y > 0 (ReLU gradient), in place on dy
__global__ void k_relu_bwd(bf16* __restrict__ dy, const bf16* __restrict__ y, long long n) {
    const bf16 zero = __float2bfloat16(0.f);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        if (!(__bfloat162float(y[i]) > 0.f)) dy[i] = zero;
}

// db[c] += sum over voxels of dy[v][c]
__global__ void k_bias_grad(const bf16* __restrict__ dy, int C, long long nv, float* __restrict__ db) {
    __shared__ float sh[256];
    const int c = blockIdx.y;
    float s = 0.f;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nv; v += (long long)gridDim.x * blockDim.x)
        s += __bfloat162float(dy[v * C + c]);
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(db + c, sh[0]);
}

// 2x2x2 average pooling: (nx,ny,nz,C) -> (nx/2,ny/2,nz/2,C)
__global__ void k_pool(const bf16* __restrict__ in, bf16* __restrict__ out, int nx, int ny, int nz, int C) {
    const int hx = nx / 2, hy = ny / 2, hz = nz / 2;
    const long long n = (long long)hx * hy * hz * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = int(i % C);
        long long v = i / C;
        const int x = int(v % hx), y = int((v / hx) % hy), z = int(v / ((long long)hx * hy));
        float s = 0.f;
        for (int q = 0; q < 8; ++q) {
            const int xx = 2 * x + (q & 1), yy = 2 * y + ((q >> 1) & 1), zz = 2 * z + (q >> 2);
            s += __bfloat162float(in[(((long long)zz * ny + yy) * nx + xx) * C + c]);
        }
        out[i] = __float2bfloat16(0.125f * s);
    }
}

// gradient of the pooling, added into din (din += dout(parent) / 8)
__global__ void k_pool_bwd(const bf16* __restrict__ dout, bf16* __restrict__ din, int nx, int ny, int nz, int C,
                           int accumulate) {
    const long long n = (long long)nx * ny * nz * C;
    const int hx = nx / 2, hy = ny / 2;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = int(i % C);
        const long long v = i / C;
        const int x = int(v % nx), y = int((v / nx) % ny), z = int(v / ((long long)nx * ny));
        const float g = 0.125f * __bfloat162float(dout[(((long long)(z / 2) * hy + y / 2) * hx + x / 2) * C + c]);
        din[i] = __float2bfloat16(accumulate ? __bfloat162float(din[i]) + g : g);
    }
}

// nearest upsampling of a (coarse, Ca channels) concatenated with b (fine, Cb channels)
__global__ void k_upcat(const bf16* __restrict__ a, int Ca, const bf16* __restrict__ b, int Cb,
                        bf16* __restrict__ out, int nx, int ny, int nz) {
    const int C = Ca + Cb, hx = nx / 2, hy = ny / 2;
    const long long n = (long long)nx * ny * nz * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = int(i % C);
        const long long v = i / C;
        if (c < Ca) {
            const int x = int(v % nx), y = int((v / nx) % ny), z = int(v / ((long long)nx * ny));
            out[i] = a[(((long long)(z / 2) * hy + y / 2) * hx + x / 2) * Ca + c];
        } else {
            out[i] = b[v * Cb + (c - Ca)];
        }
    }
}

// gradient of upcat: da (coarse) = sum of the 8 children's first Ca channels; db += last Cb
__global__ void k_upcat_bwd_a(const bf16* __restrict__ dcat, int Ca, int Cb, bf16* __restrict__ da, int nx, int ny,
                              int nz) {
    const int C = Ca + Cb, hx = nx / 2, hy = ny / 2, hz = nz / 2;
    const long long n = (long long)hx * hy * hz * Ca;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = int(i % Ca);
        const long long v = i / Ca;
        const int x = int(v % hx), y = int((v / hx) % hy), z = int(v / ((long long)hx * hy));
        float s = 0.f;
        for (int q = 0; q < 8; ++q) {
            const int xx = 2 * x + (q & 1), yy = 2 * y + ((q >> 1) & 1), zz = 2 * z + (q >> 2);
            s += __bfloat162float(dcat[(((long long)zz * ny + yy) * nx + xx) * C + c]);
        }
        da[i] = __float2bfloat16(s);
    }
}
__global__ void k_upcat_bwd_b(const bf16* __restrict__ dcat, int Ca, int Cb, bf16* __restrict__ db, long long nv) {
    const int C = Ca + Cb;
    const long long n = nv * Cb;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long v = i / Cb;
        const int c = int(i % Cb);
        db[i] = __float2bfloat16(__bfloat162float(db[i]) + __bfloat162float(dcat[v * C + Ca + c]));
    }
}

// Adam on FP32 masters (Kingma & Ba, 2015), bias-corrected step size lr_t
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       long long n, float lr_t, float b1, float b2, float eps) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr_t * mi / (sqrtf(vi) + eps);
    }
}

// geometry channels: F, mean x/y/z aperture of the cell, log of the spacing ratios
__global__ void k_geometry(vofp::Dims d, const double* __restrict__ F, const double* __restrict__ axe,
                           const double* __restrict__ aye, const double* __restrict__ aze,
                           const double* __restrict__ dx, const double* __restrict__ dy, const double* __restrict__ dz,
                           double dxmin, double dymin, double dzmin, const int32_t* __restrict__ root,
                           bf16* __restrict__ geo, float* __restrict__ mask) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < d.n; c += (long long)gridDim.x * blockDim.x) {
        const unsigned int uc = (unsigned int)c, nx = (unsigned int)d.nx, ny = (unsigned int)d.ny;
        const unsigned int tq = uc / nx;
        const int i = int(uc - tq * nx), j = int(tq % ny), k = int(tq / ny);
        const long long fx = i + (long long)(d.nx + 1) * (j + (long long)d.ny * k);
        const long long fy = i + (long long)d.nx * (j + (long long)(d.ny + 1) * k);
        const long long fz = c;
        bf16* o = geo + c * 8;
        o[0] = __float2bfloat16((float)F[c]);
        o[1] = __float2bfloat16((float)(0.5 * (axe[fx] + axe[fx + 1])));
        o[2] = __float2bfloat16((float)(0.5 * (aye[fy] + aye[fy + d.nx])));
        o[3] = __float2bfloat16((float)(0.5 * (aze[fz] + aze[fz + d.plane])));
        o[4] = __float2bfloat16((float)log(dx[i] / dxmin));
        o[5] = __float2bfloat16((float)log(dy[j] / dymin));
        o[6] = __float2bfloat16((float)log(dz[k] / dzmin));
        o[7] = __float2bfloat16(0.f);
        mask[c] = root[c] >= 0 ? 1.f : 0.f;
    }
}

}  // namespace nn
}  // namespace vofp

// =============================================================================================
// Network object
// =============================================================================================
namespace {

using vofp::nn::bf16;

struct Layer {
    int cin, cout, cin_real;
    float *w = nullptr, *b = nullptr, *gw = nullptr, *gb = nullptr;
    float *mw = nullptr, *vw = nullptr, *mb = nullptr, *vb = nullptr;
    bf16 *wb = nullptr, *wt = nullptr;
    long long nw() const { return 27LL * cout * cin; }
};

// encoder 1, 2, 3, decoder 2, 1 (two 3x3x3 convolutions each)
const int kLayers[10][3] = {{16, 16, 8},  {16, 16, 16}, {16, 32, 16}, {32, 32, 32}, {32, 64, 32},
                            {64, 64, 64}, {96, 32, 96}, {32, 32, 32}, {48, 16, 48}, {16, 16, 16}};

}  // namespace

struct vofp_nn {
    cudaStream_t stream = nullptr;
    std::string err;
    std::vector<Layer> L;
    float *hw = nullptr, *hb = nullptr, *ghw = nullptr, *ghb = nullptr;
    float *mhw = nullptr, *vhw = nullptr, *mhb = nullptr, *vhb = nullptr;
    long long nparams = 0;
    int step = 0;
    std::vector<void*> allocs;
    size_t bytes = 0;
    // grid-dependent
    int nx = 0, ny = 0, nz = 0;
    long long V1 = 0, V2 = 0, V3 = 0;
    std::vector<void*> grid_allocs;
    bf16 *geo = nullptr, *x0 = nullptr, *a1 = nullptr, *s1 = nullptr, *p1 = nullptr, *a2 = nullptr, *s2 = nullptr;
    bf16 *p2 = nullptr, *a3 = nullptr, *b3 = nullptr, *c2 = nullptr, *d2a = nullptr, *d2b = nullptr, *c1 = nullptr;
    bf16 *d1a = nullptr, *d1b = nullptr;
    bf16 *g16a = nullptr, *g16b = nullptr, *g48 = nullptr, *g32a = nullptr, *g32b = nullptr, *g96 = nullptr;
    bf16 *g64a = nullptr, *g64b = nullptr, *gs1 = nullptr, *gs2 = nullptr, *gp1 = nullptr, *gp2 = nullptr;
    float *mask = nullptr, *out = nullptr, *scal = nullptr;   // scal: sum r^2, count, scale, inv scale, loss
    bool bound = false;

    template <typename T>
    vofp_status alloc(T** p, size_t count, bool grid) {
        void* q = nullptr;
        if (cudaMalloc(&q, sizeof(T) * (count ? count : 1)) != cudaSuccess) {
            err = "cudaMalloc failed";
            return VOFP_ERR_OOM;
        }
        (grid ? grid_allocs : allocs).push_back(q);
        bytes += sizeof(T) * count;
        *p = reinterpret_cast<T*>(q);
        return VOFP_OK;
    }
};

namespace vofp {
namespace nn {
namespace {

int gs(long long n, int threads = 256) {
    long long b = (n + threads - 1) / threads;
    return (int)std::max(1LL, std::min(b, (long long)num_sms() * 16));
}

// r.r over cells with an unknown, and their count, into scal[0], scal[1]; then scale = rms
__global__ void k_rms(const float* __restrict__ r, const float* __restrict__ mask, long long n, float* scal) {
    __shared__ float sh[2][256];
    float s = 0.f, c = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        s += mask[i] * r[i] * r[i];
        c += mask[i];
    }
    sh[0][threadIdx.x] = s;
    sh[1][threadIdx.x] = c;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + o];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        atomicAdd(scal, sh[0][0]);
        atomicAdd(scal + 1, sh[1][0]);
    }
}
__global__ void k_rms_finish(float* scal) {
    const float rms = scal[1] > 0.f ? sqrtf(scal[0] / scal[1]) : 0.f;
    scal[2] = rms;
    scal[3] = rms > 0.f ? 1.f / rms : 0.f;
}
__global__ void k_pack_input_dev(const bf16* __restrict__ geo, const float* __restrict__ r, const float* scal,
                                 bf16* __restrict__ x, long long nv) {
    const float inv = scal[3];
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nv; v += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < 7; ++c) x[v * 16 + c] = geo[v * 8 + c];
        x[v * 16 + 7] = __float2bfloat16(r[v] * inv);
#pragma unroll
        for (int c = 8; c < 16; ++c) x[v * 16 + c] = __float2bfloat16(0.f);
    }
}
__global__ void k_head_dev(const bf16* __restrict__ h, const float* __restrict__ w, const float* __restrict__ b,
                           const float* scal, const float* __restrict__ mask, float* __restrict__ out, long long nv) {
    const float scale = scal[2];
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nv; v += (long long)gridDim.x * blockDim.x) {
        float s = b[0];
#pragma unroll
        for (int c = 0; c < 16; ++c) s = fmaf(w[c], __bfloat162float(h[v * 16 + c]), s);
        out[v] = mask[v] * s * scale;
    }
}
__global__ void k_head_bwd_dev(const bf16* __restrict__ h, const float* __restrict__ w, const float* __restrict__ out,
                               const float* __restrict__ target, const float* __restrict__ mask, float* scal,
                               bf16* __restrict__ dh, float* __restrict__ dw, float* __restrict__ db, long long nv) {
    __shared__ float sh[18][128];
    const float inv_scale = scal[3], inv_count = scal[1] > 0.f ? 1.f / scal[1] : 0.f;
    float lw[16], lb = 0.f, ll = 0.f;
#pragma unroll
    for (int c = 0; c < 16; ++c) lw[c] = 0.f;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nv; v += (long long)gridDim.x * blockDim.x) {
        const float e = mask[v] * (out[v] - target[v]) * inv_scale;
        ll += e * e;
        const float go = 2.f * e * inv_count;
        lb += go;
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            lw[c] = fmaf(go, __bfloat162float(h[v * 16 + c]), lw[c]);
            dh[v * 16 + c] = __float2bfloat16(go * w[c]);
        }
    }
#pragma unroll
    for (int c = 0; c < 16; ++c) sh[c][threadIdx.x] = lw[c];
    sh[16][threadIdx.x] = lb;
    sh[17][threadIdx.x] = ll;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int c = 0; c < 18; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x < 16) atomicAdd(dw + threadIdx.x, sh[threadIdx.x][0]);
    if (threadIdx.x == 16) atomicAdd(db, sh[16][0]);
    if (threadIdx.x == 17) atomicAdd(scal + 4, sh[17][0] * inv_count);
}

void conv_fwd(vofp_nn* n, const bf16* in, int cin, const Layer& l, bf16* out, int nx, int ny, int nz, bool relu,
              bool transposed_weights, int cout_override) {
    const int cout = transposed_weights ? cout_override : l.cout;
    const bf16* w = transposed_weights ? l.wt : l.wb;
    const float* bias = transposed_weights ? nullptr : l.b;
    dim3 grid((nx + 63) / 64, ny, nz);
    cudaStream_t st = n->stream;
    const int r = relu ? 1 : 0;
    switch (cout) {
        case 16: k_conv3<16><<<grid, 128, 0, st>>>(in, cin, w, bias, out, nx, ny, nz, r); break;
        case 32: k_conv3<32><<<grid, 128, 0, st>>>(in, cin, w, bias, out, nx, ny, nz, r); break;
        case 48: k_conv3<48><<<grid, 128, 0, st>>>(in, cin, w, bias, out, nx, ny, nz, r); break;
        case 64: k_conv3<64><<<grid, 128, 0, st>>>(in, cin, w, bias, out, nx, ny, nz, r); break;
        case 96: k_conv3<96><<<grid, 128, 0, st>>>(in, cin, w, bias, out, nx, ny, nz, r); break;
        default: break;
    }
}

void conv_wgrad(vofp_nn* n, const bf16* x, const bf16* dy, const Layer& l, int nx, int ny, int nz) {
    const long long rows = (long long)ny * nz;
    const int bx = 27 * (l.cout / 16);
    const long long by = std::max(1LL, std::min(rows, (long long)num_sms() * 8 / bx + 1));
    const int rpb = (int)((rows + by - 1) / by);
    dim3 grid(bx, (unsigned)((rows + rpb - 1) / rpb));
    cudaStream_t st = n->stream;
    switch (l.cin) {
        case 16: k_conv3_wgrad<16><<<grid, 128, 0, st>>>(x, dy, l.cout, l.gw, nx, ny, nz, rpb); break;
        case 32: k_conv3_wgrad<32><<<grid, 128, 0, st>>>(x, dy, l.cout, l.gw, nx, ny, nz, rpb); break;
        case 48: k_conv3_wgrad<48><<<grid, 128, 0, st>>>(x, dy, l.cout, l.gw, nx, ny, nz, rpb); break;
        case 64: k_conv3_wgrad<64><<<grid, 128, 0, st>>>(x, dy, l.cout, l.gw, nx, ny, nz, rpb); break;
        case 96: k_conv3_wgrad<96><<<grid, 128, 0, st>>>(x, dy, l.cout, l.gw, nx, ny, nz, rpb); break;
        default: break;
    }
    const long long nv = (long long)nx * ny * nz;
    k_bias_grad<<<dim3(gs(nv), l.cout), 256, 0, st>>>(dy, l.cout, nv, l.gb);
}

void refresh_bf16(vofp_nn* n) {
    for (auto& l : n->L) k_weights_bf16<<<gs(l.nw()), 256, 0, n->stream>>>(l.w, l.wb, l.wt, l.cout, l.cin);
}

vofp_status forward(vofp_nn* n, const float* r) {
    cudaStream_t st = n->stream;
    const int X = n->nx, Y = n->ny, Z = n->nz;
    cudaMemsetAsync(n->scal, 0, sizeof(float) * 8, st);
    k_rms<<<gs(n->V1), 256, 0, st>>>(r, n->mask, n->V1, n->scal);
    k_rms_finish<<<1, 1, 0, st>>>(n->scal);
    k_pack_input_dev<<<gs(n->V1), 256, 0, st>>>(n->geo, r, n->scal, n->x0, n->V1);
    auto& L = n->L;
    conv_fwd(n, n->x0, 16, L[0], n->a1, X, Y, Z, true, false, 0);
    conv_fwd(n, n->a1, 16, L[1], n->s1, X, Y, Z, true, false, 0);
    k_pool<<<gs(n->V2 * 16), 256, 0, st>>>(n->s1, n->p1, X, Y, Z, 16);
    conv_fwd(n, n->p1, 16, L[2], n->a2, X / 2, Y / 2, Z / 2, true, false, 0);
    conv_fwd(n, n->a2, 32, L[3], n->s2, X / 2, Y / 2, Z / 2, true, false, 0);
    k_pool<<<gs(n->V3 * 32), 256, 0, st>>>(n->s2, n->p2, X / 2, Y / 2, Z / 2, 32);
    conv_fwd(n, n->p2, 32, L[4], n->a3, X / 4, Y / 4, Z / 4, true, false, 0);
    conv_fwd(n, n->a3, 64, L[5], n->b3, X / 4, Y / 4, Z / 4, true, false, 0);
    k_upcat<<<gs(n->V2 * 96), 256, 0, st>>>(n->b3, 64, n->s2, 32, n->c2, X / 2, Y / 2, Z / 2);
    conv_fwd(n, n->c2, 96, L[6], n->d2a, X / 2, Y / 2, Z / 2, true, false, 0);
    conv_fwd(n, n->d2a, 32, L[7], n->d2b, X / 2, Y / 2, Z / 2, true, false, 0);
    k_upcat<<<gs(n->V1 * 48), 256, 0, st>>>(n->d2b, 32, n->s1, 16, n->c1, X, Y, Z);
    conv_fwd(n, n->c1, 48, L[8], n->d1a, X, Y, Z, true, false, 0);
    conv_fwd(n, n->d1a, 16, L[9], n->d1b, X, Y, Z, true, false, 0);
    k_head_dev<<<gs(n->V1), 256, 0, st>>>(n->d1b, n->hw, n->hb, n->scal, n->mask, n->out, n->V1);
    return cudaGetLastError() == cudaSuccess ? VOFP_OK : VOFP_ERR_CUDA;
}

// gradient of one conv layer y = relu(conv(x)): dy (BF16, in place -> dpre), weight/bias grads,
// and optionally the input gradient dx
void layer_bwd(vofp_nn* n, const Layer& l, const bf16* x, const bf16* y, bf16* dy, bf16* dx, int nx, int ny, int nz) {
    const long long nv = (long long)nx * ny * nz;
    k_relu_bwd<<<gs(nv * l.cout), 256, 0, n->stream>>>(dy, y, nv * l.cout);
    conv_wgrad(n, x, dy, l, nx, ny, nz);
    if (dx) conv_fwd(n, dy, l.cout, l, dx, nx, ny, nz, false, true, l.cin);
}

vofp_status backward(vofp_nn* n, const float* target) {
    cudaStream_t st = n->stream;
    const int X = n->nx, Y = n->ny, Z = n->nz;
    const int X2 = X / 2, Y2 = Y / 2, Z2 = Z / 2, X4 = X / 4, Y4 = Y / 4, Z4 = Z / 4;
    auto& L = n->L;
    for (auto& l : L) {
        cudaMemsetAsync(l.gw, 0, sizeof(float) * l.nw(), st);
        cudaMemsetAsync(l.gb, 0, sizeof(float) * l.cout, st);
    }
    cudaMemsetAsync(n->ghw, 0, sizeof(float) * 16, st);
    cudaMemsetAsync(n->ghb, 0, sizeof(float), st);
    k_head_bwd_dev<<<gs(n->V1, 128), 128, 0, st>>>(n->d1b, n->hw, n->out, target, n->mask, n->scal, n->g16a, n->ghw,
                                                   n->ghb, n->V1);
    layer_bwd(n, L[9], n->d1a, n->d1b, n->g16a, n->g16b, X, Y, Z);           // -> d(d1a)
    layer_bwd(n, L[8], n->c1, n->d1a, n->g16b, n->g48, X, Y, Z);             // -> d(c1)
    cudaMemsetAsync(n->gs1, 0, sizeof(bf16) * n->V1 * 16, st);
    k_upcat_bwd_a<<<gs(n->V2 * 32), 256, 0, st>>>(n->g48, 32, 16, n->g32a, X, Y, Z);   // -> d(d2b)
    k_upcat_bwd_b<<<gs(n->V1 * 16), 256, 0, st>>>(n->g48, 32, 16, n->gs1, n->V1);      // skip 1
    layer_bwd(n, L[7], n->d2a, n->d2b, n->g32a, n->g32b, X2, Y2, Z2);        // -> d(d2a)
    layer_bwd(n, L[6], n->c2, n->d2a, n->g32b, n->g96, X2, Y2, Z2);          // -> d(c2)
    cudaMemsetAsync(n->gs2, 0, sizeof(bf16) * n->V2 * 32, st);
    k_upcat_bwd_a<<<gs(n->V3 * 64), 256, 0, st>>>(n->g96, 64, 32, n->g64a, X2, Y2, Z2);  // -> d(b3)
    k_upcat_bwd_b<<<gs(n->V2 * 32), 256, 0, st>>>(n->g96, 64, 32, n->gs2, n->V2);       // skip 2
    layer_bwd(n, L[5], n->a3, n->b3, n->g64a, n->g64b, X4, Y4, Z4);          // -> d(a3)
    layer_bwd(n, L[4], n->p2, n->a3, n->g64b, n->gp2, X4, Y4, Z4);           // -> d(p2)
    k_pool_bwd<<<gs(n->V2 * 32), 256, 0, st>>>(n->gp2, n->gs2, X2, Y2, Z2, 32, 1);
    layer_bwd(n, L[3], n->a2, n->s2, n->gs2, n->g32a, X2, Y2, Z2);           // -> d(a2)
    layer_bwd(n, L[2], n->p1, n->a2, n->g32a, n->gp1, X2, Y2, Z2);           // -> d(p1)
    k_pool_bwd<<<gs(n->V1 * 16), 256, 0, st>>>(n->gp1, n->gs1, X, Y, Z, 16, 1);
    layer_bwd(n, L[1], n->a1, n->s1, n->gs1, n->g16a, X, Y, Z);              // -> d(a1)
    layer_bwd(n, L[0], n->x0, n->a1, n->g16a, nullptr, X, Y, Z);
    return cudaGetLastError() == cudaSuccess ? VOFP_OK : VOFP_ERR_CUDA;
}

void adam(vofp_nn* n, float lr) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    n->step += 1;
    const float lr_t = lr * std::sqrt(1.f - std::pow(b2, (float)n->step)) / (1.f - std::pow(b1, (float)n->step));
    for (auto& l : n->L) {
        k_adam<<<gs(l.nw()), 256, 0, n->stream>>>(l.w, l.gw, l.mw, l.vw, l.nw(), lr_t, b1, b2, eps);
        k_adam<<<1, 64, 0, n->stream>>>(l.b, l.gb, l.mb, l.vb, l.cout, lr_t, b1, b2, eps);
    }
    k_adam<<<1, 32, 0, n->stream>>>(n->hw, n->ghw, n->mhw, n->vhw, 16, lr_t, b1, b2, eps);
    k_adam<<<1, 32, 0, n->stream>>>(n->hb, n->ghb, n->mhb, n->vhb, 1, lr_t, b1, b2, eps);
    refresh_bf16(n);
}

vofp_status ensure_grid(vofp_nn* n, int nx, int ny, int nz) {
    if (nx % 4 || ny % 4 || nz % 4 || nx < 4 || ny < 4 || nz < 4) {
        n->err = "grid sizes must be positive multiples of 4 (two 2x2x2 poolings)";
        return VOFP_ERR_INVALID_ARG;
    }
    if (n->bound && n->nx == nx && n->ny == ny && n->nz == nz) return VOFP_OK;
    cudaStreamSynchronize(n->stream);
    for (void* p : n->grid_allocs) cudaFree(p);
    n->grid_allocs.clear();
    n->nx = nx;
    n->ny = ny;
    n->nz = nz;
    n->V1 = (long long)nx * ny * nz;
    n->V2 = n->V1 / 8;
    n->V3 = n->V1 / 64;
    const long long V1 = n->V1, V2 = n->V2, V3 = n->V3;
    vofp_status s;
    if ((s = n->alloc(&n->geo, V1 * 8, true)) || (s = n->alloc(&n->x0, V1 * 16, true)) ||
        (s = n->alloc(&n->a1, V1 * 16, true)) || (s = n->alloc(&n->s1, V1 * 16, true)) ||
        (s = n->alloc(&n->p1, V2 * 16, true)) || (s = n->alloc(&n->a2, V2 * 32, true)) ||
        (s = n->alloc(&n->s2, V2 * 32, true)) || (s = n->alloc(&n->p2, V3 * 32, true)) ||
        (s = n->alloc(&n->a3, V3 * 64, true)) || (s = n->alloc(&n->b3, V3 * 64, true)) ||
        (s = n->alloc(&n->c2, V2 * 96, true)) || (s = n->alloc(&n->d2a, V2 * 32, true)) ||
        (s = n->alloc(&n->d2b, V2 * 32, true)) || (s = n->alloc(&n->c1, V1 * 48, true)) ||
        (s = n->alloc(&n->d1a, V1 * 16, true)) || (s = n->alloc(&n->d1b, V1 * 16, true)) ||
        (s = n->alloc(&n->g16a, V1 * 16, true)) || (s = n->alloc(&n->g16b, V1 * 16, true)) ||
        (s = n->alloc(&n->g48, V1 * 48, true)) || (s = n->alloc(&n->g32a, V2 * 32, true)) ||
        (s = n->alloc(&n->g32b, V2 * 32, true)) || (s = n->alloc(&n->g96, V2 * 96, true)) ||
        (s = n->alloc(&n->g64a, V3 * 64, true)) || (s = n->alloc(&n->g64b, V3 * 64, true)) ||
        (s = n->alloc(&n->gs1, V1 * 16, true)) || (s = n->alloc(&n->gs2, V2 * 32, true)) ||
        (s = n->alloc(&n->gp1, V2 * 16, true)) || (s = n->alloc(&n->gp2, V3 * 32, true)) ||
        (s = n->alloc(&n->mask, V1, true)) || (s = n->alloc(&n->out, V1, true)))
        return s;
    n->bound = true;
    return VOFP_OK;
}

std::vector<std::pair<float*, long long>> param_list(vofp_nn* n, bool grads) {
    std::vector<std::pair<float*, long long>> v;
    for (auto& l : n->L) {
        v.push_back({grads ? l.gw : l.w, l.nw()});
        v.push_back({grads ? l.gb : l.b, l.cout});
    }
    v.push_back({grads ? n->ghw : n->hw, 16});
    v.push_back({grads ? n->ghb : n->hb, 1});
    return v;
}

}  // namespace
}  // namespace nn
}  // namespace vofp

using namespace vofp::nn;

namespace vofp {
namespace nn {
long long bound_cells(const vofp_nn* n) { return n && n->bound ? n->V1 : -1; }
cudaStream_t stream_of(const vofp_nn* n) { return n ? n->stream : nullptr; }
}  // namespace nn
}  // namespace vofp

extern "C" {

vofp_status vofp_nn_create(vofp_nn** out, unsigned long long seed, vofp_stream stream) {
    if (!out) return VOFP_ERR_INVALID_ARG;
    *out = nullptr;
    vofp_nn* n = new (std::nothrow) vofp_nn();
    if (!n) return VOFP_ERR_OOM;
    n->stream = reinterpret_cast<cudaStream_t>(stream);
    std::mt19937_64 rng(seed);
    vofp_status s;
    for (int i = 0; i < 10; ++i) {
        Layer l;
        l.cin = kLayers[i][0];
        l.cout = kLayers[i][1];
        l.cin_real = kLayers[i][2];
        if ((s = n->alloc(&l.w, l.nw(), false)) || (s = n->alloc(&l.b, l.cout, false)) ||
            (s = n->alloc(&l.gw, l.nw(), false)) || (s = n->alloc(&l.gb, l.cout, false)) ||
            (s = n->alloc(&l.mw, l.nw(), false)) || (s = n->alloc(&l.vw, l.nw(), false)) ||
            (s = n->alloc(&l.mb, l.cout, false)) || (s = n->alloc(&l.vb, l.cout, false)) ||
            (s = n->alloc(&l.wb, l.nw(), false)) || (s = n->alloc(&l.wt, l.nw(), false))) {
            vofp_nn_destroy(n);
            return s;
        }
        // He initialisation over the real fan-in; padded input channels start (and stay) at 0
        std::normal_distribution<float> nd(0.f, std::sqrt(2.f / (27.f * l.cin_real)));
        std::vector<float> hw(l.nw());
        for (long long q = 0; q < l.nw(); ++q) hw[q] = (q % l.cin) < l.cin_real ? nd(rng) : 0.f;
        std::vector<float> zb(l.cout, 0.f);
        cudaMemcpy(l.w, hw.data(), sizeof(float) * l.nw(), cudaMemcpyHostToDevice);
        cudaMemcpy(l.b, zb.data(), sizeof(float) * l.cout, cudaMemcpyHostToDevice);
        cudaMemset(l.mw, 0, sizeof(float) * l.nw());
        cudaMemset(l.vw, 0, sizeof(float) * l.nw());
        cudaMemset(l.mb, 0, sizeof(float) * l.cout);
        cudaMemset(l.vb, 0, sizeof(float) * l.cout);
        n->nparams += l.nw() + l.cout;
        n->L.push_back(l);
    }
    if ((s = n->alloc(&n->hw, 16, false)) || (s = n->alloc(&n->hb, 1, false)) || (s = n->alloc(&n->ghw, 16, false)) ||
        (s = n->alloc(&n->ghb, 1, false)) || (s = n->alloc(&n->mhw, 16, false)) || (s = n->alloc(&n->vhw, 16, false)) ||
        (s = n->alloc(&n->mhb, 1, false)) || (s = n->alloc(&n->vhb, 1, false)) || (s = n->alloc(&n->scal, 8, false))) {
        vofp_nn_destroy(n);
        return s;
    }
    std::normal_distribution<float> nh(0.f, std::sqrt(1.f / 16.f));
    float hw[16], hb = 0.f;
    for (auto& v : hw) v = nh(rng);
    cudaMemcpy(n->hw, hw, sizeof(hw), cudaMemcpyHostToDevice);
    cudaMemcpy(n->hb, &hb, sizeof(float), cudaMemcpyHostToDevice);
    cudaMemset(n->mhw, 0, 16 * sizeof(float));
    cudaMemset(n->vhw, 0, 16 * sizeof(float));
    cudaMemset(n->mhb, 0, sizeof(float));
    cudaMemset(n->vhb, 0, sizeof(float));
    n->nparams += 17;
    refresh_bf16(n);
    if (cudaStreamSynchronize(n->stream) != cudaSuccess) {
        vofp_nn_destroy(n);
        return VOFP_ERR_CUDA;
    }
    *out = n;
    return VOFP_OK;
}

void vofp_nn_destroy(vofp_nn* n) {
    if (!n) return;
    cudaStreamSynchronize(n->stream);
    for (void* p : n->grid_allocs) cudaFree(p);
    for (void* p : n->allocs) cudaFree(p);
    delete n;
}

const char* vofp_nn_last_error(const vofp_nn* n) { return n ? n->err.c_str() : "null network"; }

vofp_status vofp_nn_param_count(const vofp_nn* n, long long* count) {
    if (!n || !count) return VOFP_ERR_INVALID_ARG;
    *count = n->nparams;
    return VOFP_OK;
}

vofp_status vofp_nn_get_params(vofp_nn* n, float* host, long long count, int grads) {
    if (!n || !host || count != n->nparams) return VOFP_ERR_INVALID_ARG;
    long long off = 0;
    for (auto& pr : param_list(n, grads != 0)) {
        if (cudaMemcpyAsync(host + off, pr.first, sizeof(float) * pr.second, cudaMemcpyDeviceToHost, n->stream) !=
            cudaSuccess)
            return VOFP_ERR_CUDA;
        off += pr.second;
    }
    return cudaStreamSynchronize(n->stream) == cudaSuccess ? VOFP_OK : VOFP_ERR_CUDA;
}

vofp_status vofp_nn_set_params(vofp_nn* n, const float* host, long long count) {
    if (!n || !host || count != n->nparams) return VOFP_ERR_INVALID_ARG;
    long long off = 0;
    for (auto& pr : param_list(n, false)) {
        if (cudaMemcpyAsync(pr.first, host + off, sizeof(float) * pr.second, cudaMemcpyHostToDevice, n->stream) !=
            cudaSuccess)
            return VOFP_ERR_CUDA;
        off += pr.second;
    }
    refresh_bf16(n);
    return cudaStreamSynchronize(n->stream) == cudaSuccess ? VOFP_OK : VOFP_ERR_CUDA;
}

vofp_status vofp_nn_bind(vofp_nn* n, vofp_ctx* c, const double* F) {
    if (!n || !c || !F) return VOFP_ERR_INVALID_ARG;
    if (!c->built) {
        n->err = "operator not built";
        return VOFP_ERR_NOT_BUILT;
    }
    vofp_status s = ensure_grid(n, c->d.nx, c->d.ny, c->d.nz);
    if (s) return s;
    const double dxmin = *std::min_element(c->hdx.begin(), c->hdx.end());
    const double dymin = *std::min_element(c->hdy.begin(), c->hdy.end());
    const double dzmin = *std::min_element(c->hdz.begin(), c->hdz.end());
    k_geometry<<<gs(c->d.n), 256, 0, n->stream>>>(c->d, F, c->axe, c->aye, c->aze, c->dx, c->dy, c->dz, dxmin, dymin,
                                                  dzmin, c->root, n->geo, n->mask);
    return cudaGetLastError() == cudaSuccess ? VOFP_OK : VOFP_ERR_CUDA;
}

vofp_status vofp_nn_export_geometry(vofp_nn* n, uint16_t* geo, float* mask) {
    if (!n || !n->bound || !geo || !mask) return VOFP_ERR_INVALID_ARG;
    cudaMemcpyAsync(geo, n->geo, sizeof(bf16) * n->V1 * 8, cudaMemcpyDeviceToDevice, n->stream);
    cudaMemcpyAsync(mask, n->mask, sizeof(float) * n->V1, cudaMemcpyDeviceToDevice, n->stream);
    return cudaGetLastError() == cudaSuccess ? VOFP_OK : VOFP_ERR_CUDA;
}

vofp_status vofp_nn_set_geometry(vofp_nn* n, int nx, int ny, int nz, const uint16_t* geo, const float* mask) {
    if (!n || !geo || !mask) return VOFP_ERR_INVALID_ARG;
    vofp_status s = ensure_grid(n, nx, ny, nz);
    if (s) return s;
    cudaMemcpyAsync(n->geo, geo, sizeof(bf16) * n->V1 * 8, cudaMemcpyDeviceToDevice, n->stream);
    cudaMemcpyAsync(n->mask, mask, sizeof(float) * n->V1, cudaMemcpyDeviceToDevice, n->stream);
    return cudaGetLastError() == cudaSuccess ? VOFP_OK : VOFP_ERR_CUDA;
}

vofp_status vofp_nn_forward(vofp_nn* n, const float* r, float* z) {
    if (!n || !r || !z) return VOFP_ERR_INVALID_ARG;
    if (!n->bound) {
        n->err = "no geometry bound";
        return VOFP_ERR_NOT_BUILT;
    }
    vofp_status s = forward(n, r);
    if (s) return s;
    cudaMemcpyAsync(z, n->out, sizeof(float) * n->V1, cudaMemcpyDeviceToDevice, n->stream);
    return cudaGetLastError() == cudaSuccess ? VOFP_OK : VOFP_ERR_CUDA;
}

vofp_status vofp_nn_train_step(vofp_nn* n, const float* r, const float* target, float lr, int update, float* loss) {
    if (!n || !r || !target) return VOFP_ERR_INVALID_ARG;
    if (!n->bound) {
        n->err = "no geometry bound";
        return VOFP_ERR_NOT_BUILT;
    }
    vofp_status s;
    if ((s = forward(n, r)) || (s = backward(n, target))) return s;
    if (update) adam(n, lr);
    if (loss) {
        if (cudaMemcpyAsync(loss, n->scal + 4, sizeof(float), cudaMemcpyDeviceToHost, n->stream) != cudaSuccess)
            return VOFP_ERR_CUDA;
        if (cudaStreamSynchronize(n->stream) != cudaSuccess) return VOFP_ERR_CUDA;
    }
    return cudaGetLastError() == cudaSuccess ? VOFP_OK : VOFP_ERR_CUDA;
}

}  // extern "C"
