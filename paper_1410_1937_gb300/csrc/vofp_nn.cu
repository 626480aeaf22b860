// Learned preconditioner: a 3-level 3-D convolutional encoder-decoder (16/32/64 channels, 3x3x3
// kernels, zero padding, ReLU, 2x2x2 average pooling, nearest upsampling, skip concatenation, a
// final 1x1x1 layer) that maps the operator's geometry and a residual to an approximate solution
// of the scaled pressure system.  The paper has no counterpart: the network is used as the
// preconditioner and initial guess of a flexible CG around the paper's conjugate-gradient solve.
//
// Activations are BF16 in a chunk-planar layout: channels in groups of eight, each group a plane
// of 16-byte voxel records, ((c / 8) * V + v) * 8 + c % 8 for voxel v of V.  A voxel's eight
// channels of one group are then one row of a tensor-core operand, a box of voxels of one group is
// one contiguous block, and concatenating channels is placing groups side by side (the skip
// connections write straight into the concatenated buffers).
//
// Every 3x3x3 convolution, forward and data gradient, is an implicit GEMM on the fifth-generation
// tensor cores (k_conv3_umma): a block owns an 8 x 16 voxel tile of a plane (M = 128) and marches
// it in z; a bulk tensor copy brings each input plane with its one-voxel halo into a ring of
// shared-memory slots; one thread issues, per output plane, 27 taps x (input channels / 16)
// tcgen05.mma instructions whose A operand is the halo'd plane shifted by the tap (a different
// descriptor start address) and whose B operand is that tap's weights, accumulating in FP32 in
// tensor memory; four warps read the accumulator back, add the bias, apply ReLU and store BF16.
// Weight gradients are tcgen05 GEMMs over the voxels with both operands read MN-major from the
// same chunk-planar tiles (k_conv3_wgrad_umma).
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <random>
#include <tuple>
#include <vector>

#include "vofp_internal.cuh"
#include "vofp_tma.cuh"
#include "vofp_umma.cuh"

namespace vofp {
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();

namespace nn {

using bf16 = __nv_bfloat16;

// channel c of voxel v in a chunk-planar tensor of V voxels
__host__ __device__ __forceinline__ long long aidx(long long v, int c, long long V) {
    return ((long long)(c >> 3) * V + v) * 8 + (c & 7);
}

// ---- 3x3x3 convolution on the tensor cores ---------------------------------------------------
// Tile of one block: 8 voxels along x (one core-matrix row group) by 16 along y (M = 128 rows,
// row m = voxel (m % 8, m / 8)); its input box is 10 x 18 voxels (one-voxel halo) of every input
// channel group.  The three z taps are columns of one instruction: input plane p times the
// weights of the three z taps (N = 3 NOUT) gives in one MMA the contributions of p to output
// planes p+1, p and p-1, which sit in consecutive TMEM column blocks (block j: z tap j, output
// p+1-j).  Output plane o therefore owns columns NOUT (S + 1 - (o - z0)) of a segment of S planes
// starting at z0 (descending in o), with one block above and two below for the contributions that
// fall outside the segment.  Each input plane is read by 9 taps x (Cin/16) MMAs and released.
constexpr int kTileX = 8, kTileY = 16, kBoxX = kTileX + 2, kBoxY = kTileY + 2;
constexpr int kGroupBytes = kBoxX * kBoxY * 16;   // one channel group of one halo'd plane
constexpr int kConvThreads = 192;                 // warp 0 copies, warp 1 issues MMAs, 2..5 store

__host__ __device__ constexpr size_t al128(size_t b) { return (b + 127) / 128 * 128; }
__host__ __device__ constexpr uint32_t pow2_at_least(uint32_t v) {
    return v <= 32 ? 32 : (v <= 64 ? 64 : (v <= 128 ? 128 : (v <= 256 ? 256 : 512)));
}

template <int CIN, int NOUT, int R>
struct ConvCfg {
    static_assert(CIN % 16 == 0 && NOUT % 16 == 0 && 3 * NOUT <= 256, "shape");
    static constexpr int KCH = CIN / 8;                               // input channel groups
    // output planes per segment: the accumulators of S + 4 planes (S outputs and the blocks that
    // fall outside the segment) in TMEM; two blocks per SM for 16 output channels, one otherwise
    static constexpr int S = NOUT == 16 ? 12 : (NOUT == 32 ? 12 : (NOUT == 48 ? 6 : 4));
    static constexpr uint32_t TCOLS = pow2_at_least((uint32_t)NOUT * (S + 4));
    static constexpr uint32_t PLANE = (uint32_t)KCH * kGroupBytes;    // bytes of one ring slot
    static constexpr uint32_t WBYTES = 27u * CIN * NOUT * 2u;         // this block's weights
    static constexpr uint32_t WTAP = (uint32_t)KCH * 3 * NOUT * 16;   // weights of one (y, x) tap
    static constexpr size_t oW = 0;
    static constexpr size_t oRing = al128(WBYTES);
    static constexpr size_t oBar = oRing + al128((size_t)R * PLANE);
    static constexpr size_t oBias = oBar + 8 * (2 * R + S + 1) + 8;
    static constexpr size_t SMEM_USED = al128(oBias + 4 * NOUT) + 128;   // + alignment slack
    // requested shared memory: at least enough to keep the blocks per SM within what tensor memory
    // holds (512 columns per SM), so that no block waits inside its TMEM allocation
    static constexpr size_t SMEM = TCOLS == 512 ? (SMEM_USED > 120 * 1024 ? SMEM_USED : 120 * 1024)
                                 : TCOLS == 256 ? (SMEM_USED > 80 * 1024 ? SMEM_USED : 80 * 1024) : SMEM_USED;
    static_assert(SMEM <= 232448, "shared memory per block");
    static_assert(TCOLS <= 512, "tensor memory");
};

struct ConvArgs {
    int nx, ny, nz;
    int tiles_x, tiles_y;
    int seg, nseg;            // planes per z segment (<= S), segments
    long long V;              // voxels of the level
    const float* bias;        // per output channel (null: none)
    int relu;
    const bf16* wblob;        // [split][9 (y, x) taps][CIN/8][3 z taps x NOUT][8]
    bf16* out;                // chunk-planar output tensor
    int out_chunk0;           // first channel group of this convolution's outputs in `out`
    int* err;                 // set to 1 when a bounded wait runs out
};

// Block order: x tiles fastest, then y tiles, z segments, output-channel splits (neighbouring
// blocks share halo rows through L2).
template <int CIN, int NOUT, int R>
__global__ void __launch_bounds__(kConvThreads, 1)
k_conv3_umma(const __grid_constant__ CUtensorMap in_map, const ConvArgs a) {
    using G = ConvCfg<CIN, NOUT, R>;
    constexpr int S = G::S;
    extern __shared__ unsigned char smraw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 127) & ~uintptr_t(127));
    unsigned char* wsm = sm + G::oW;
    unsigned char* ring = sm + G::oRing;
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + G::oBar);
    uint64_t* empty = full + R;
    uint64_t* accf = empty + R;   // one per output plane of the segment
    uint64_t* wbar = accf + S;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(wbar + 1);
    float* bsm = reinterpret_cast<float*>(sm + G::oBias);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int b = blockIdx.x;
    const int tx = b % a.tiles_x;
    b /= a.tiles_x;
    const int ty = b % a.tiles_y;
    b /= a.tiles_y;
    const int sg = b % a.nseg, split = b / a.nseg;
    const int x0 = tx * kTileX, y0 = ty * kTileY;
    const int z0 = sg * a.seg;
    const int nout = min(a.nz, z0 + a.seg) - z0;   // output planes of this block (1 .. S)
    const int nin = nout + 2;                       // input planes z0-1 .. z0+nout
    if (tid == 0) {
        for (int i = 0; i < R; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < S; ++i) mbar_init(&accf[i], 1);
        mbar_init(wbar, 1);
        fence_mbar_init();
    }
    if (tid < NOUT) bsm[tid] = a.bias ? a.bias[split * NOUT + tid] : 0.f;
    if (warp == 0) umma::tmem_alloc(tslot, G::TCOLS);
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = *tslot;
    bool fail = false;

    if (warp == 0) {
        if (lane == 0) {
            // producer: the block's weights once, then the input planes through the ring
            mbar_expect_tx(wbar, G::WBYTES);
            umma::bulk_load(wsm, reinterpret_cast<const unsigned char*>(a.wblob) + (size_t)split * G::WBYTES,
                            G::WBYTES, wbar);
            int issued = 0;
            for (int lp = 0; lp < nin; ++lp) {
                const int s = lp % R;
                if (lp >= R && !mbar_wait_bounded(&empty[s], (uint32_t)((lp / R) - 1) & 1u)) {
                    fail = true;
                    break;
                }
                mbar_expect_tx(&full[s], G::PLANE);
                umma::tma_load_5d(ring + (size_t)s * G::PLANE, &in_map, &full[s], 0, x0 - 1, y0 - 1, z0 - 1 + lp, 0);
                ++issued;
            }
            // every copy issued must have landed before the block may leave
            for (int lp = max(0, issued - R); lp < issued; ++lp)
                if (!mbar_wait_bounded(&full[lp % R], (uint32_t)(lp / R) & 1u)) fail = true;
            if (!mbar_wait_bounded(wbar, 0)) fail = true;
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t id1 = umma::idesc_bf16(128, NOUT), id2 = umma::idesc_bf16(128, 2 * NOUT),
                               id3 = umma::idesc_bf16(128, 3 * NOUT);
            const uint32_t wbase = umma::saddr(wsm), rbase = umma::saddr(ring);
            if (!mbar_wait_bounded(wbar, 0)) fail = true;
            for (int lp = 0; lp < nin && !fail; ++lp) {
                const int s = lp % R;
                if (!mbar_wait_bounded(&full[s], (uint32_t)(lp / R) & 1u)) {
                    fail = true;
                    break;
                }
                umma::fence_after_sync();
                // input plane z0-1+lp: block j of the result is output plane z0+lp-j
                const uint32_t d = tmem + (uint32_t)(NOUT * (S + 1 - lp));
                const uint32_t slot = rbase + (uint32_t)s * G::PLANE;
#pragma unroll 1
                for (int t = 0; t < 9; ++t) {
                    const int dy = t / 3, dx = t % 3;
                    const uint32_t abase = slot + (uint32_t)(dy * kBoxX + dx) * 16u;
                    const uint32_t bbase = wbase + (uint32_t)t * G::WTAP;
#pragma unroll
                    for (int ks = 0; ks < CIN / 16; ++ks) {
                        const uint64_t ad = umma::smem_desc(abase + 2u * ks * kGroupBytes, kGroupBytes, kBoxX * 16);
                        const uint32_t bk = bbase + 2u * ks * (3 * NOUT * 16);
                        if (t == 0 && ks == 0) {
                            // block 0 starts output plane z0+lp afresh; blocks 1, 2 add to planes
                            // that earlier input planes began
                            umma::mma_bf16(d, ad, umma::smem_desc(bk, 3 * NOUT * 16, 128), id1, 0u);
                            umma::mma_bf16(d + NOUT, ad, umma::smem_desc(bk + (NOUT / 8) * 128, 3 * NOUT * 16, 128),
                                           id2, 1u);
                        } else {
                            umma::mma_bf16(d, ad, umma::smem_desc(bk, 3 * NOUT * 16, 128), id3, 1u);
                        }
                    }
                }
                umma::commit(&empty[s]);                     // the plane's slot may be refilled
                if (lp >= 2) umma::commit(&accf[lp - 2]);    // output plane z0+lp-2 is complete
            }
        }
    } else {
        // epilogue: TMEM lane quadrant (warp % 4) of the 128 rows; row m = voxel (m % 8, m / 8)
        const int q = warp & 3;
        const int m = q * 32 + lane;
        const int xi = x0 + (m & 7), yi = y0 + (m >> 3);
        const bool inside = xi < a.nx && yi < a.ny;
        for (int lz = 0; lz < nout; ++lz) {
            if (!fail && !mbar_wait_bounded(&accf[lz], 0u)) fail = true;
            if (__any_sync(0xffffffffu, fail)) {
                fail = true;
                break;
            }
            umma::fence_after_sync();
            const uint32_t col = (uint32_t)(NOUT * (S + 1 - lz));
            float v[NOUT];
#pragma unroll
            for (int c0 = 0; c0 < NOUT; c0 += 16) {
                uint32_t r[16];
                umma::tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + col + c0, r);
                umma::tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 16; ++j) v[c0 + j] = __uint_as_float(r[j]);
            }
            if (inside) {
                const long long vox = ((long long)(z0 + lz) * a.ny + yi) * a.nx + xi;
#pragma unroll
                for (int oc = 0; oc < NOUT / 8; ++oc) {
                    uint32_t w4[4];
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        float lo = v[oc * 8 + 2 * h] + bsm[oc * 8 + 2 * h];
                        float hi = v[oc * 8 + 2 * h + 1] + bsm[oc * 8 + 2 * h + 1];
                        if (a.relu) {
                            lo = fmaxf(lo, 0.f);
                            hi = fmaxf(hi, 0.f);
                        }
                        const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
                        w4[h] = *reinterpret_cast<const uint32_t*>(&p);
                    }
                    const long long grp = a.out_chunk0 + (long long)split * (NOUT / 8) + oc;
                    *reinterpret_cast<uint4*>(a.out + (grp * a.V + vox) * 8) = make_uint4(w4[0], w4[1], w4[2], w4[3]);
                }
            }
        }
    }
    if (fail) atomicExch(a.err, 1);
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        umma::fence_after_sync();
        umma::tmem_dealloc(tmem, G::TCOLS);
    }
}

// ---- weight blobs for the tensor-core convolution ---------------------------------------------
// forward: blob[s][t][k][j nout + n][e] = W[9 j + t][s nout + n][8 k + e]  (W[27][cout][cin], FP32
// masters; t = (y, x) tap, j = z tap)
__global__ void k_blob_fwd(const float* __restrict__ w, int cout, int cin, int nout, bf16* __restrict__ blob) {
    const long long total = 27LL * cout * cin;
    const int kch = cin / 8;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        long long q = i;
        const int e = int(q & 7);
        q >>= 3;
        const int jn = int(q % (3 * nout));
        q /= 3 * nout;
        const int k = int(q % kch);
        q /= kch;
        const int t = int(q % 9);
        const int s = int(q / 9);
        const int j = jn / nout, n = jn % nout;
        blob[i] = __float2bfloat16(w[((long long)(9 * j + t) * cout + s * nout + n) * cin + 8 * k + e]);
    }
}
// data gradient: the layer run backwards (inputs: its cout channels; outputs: its cin channels;
// taps mirrored): blob[s][t][k][j nout + n][e] = W[26 - (9 j + t)][8 k + e][s nout + n]
__global__ void k_blob_dgrad(const float* __restrict__ w, int cout, int cin, int nout, bf16* __restrict__ blob) {
    const long long total = 27LL * cout * cin;
    const int kch = cout / 8;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        long long q = i;
        const int e = int(q & 7);
        q >>= 3;
        const int jn = int(q % (3 * nout));
        q /= 3 * nout;
        const int k = int(q % kch);
        q /= kch;
        const int t = int(q % 9);
        const int s = int(q / 9);
        const int j = jn / nout, n = jn % nout;
        blob[i] = __float2bfloat16(w[((long long)(26 - (9 * j + t)) * cout + 8 * k + e) * cin + s * nout + n]);
    }
}

// ---- 3x3x3 convolution, weight gradient, on the tensor cores ----------------------------------
// dW[tap][co][ci] = sum over voxels v of dy[v][co] x[v + tap - 1][ci].  Per (y, x) tap it is one
// GEMM over the voxels, D[(z tap, ci)][co] = sum_k A[(z tap, ci)][k] B[co][k] with K = voxels: A is
// the input x at the three planes z-1, z, z+1 shifted by the (y, x) tap and B the output gradient
// dy at plane z, both read MN-major straight from their chunk-planar tiles (a row of a core matrix
// is one voxel's 8 channels of a group, consecutive rows are consecutive voxels along x).  The
// input box of a tile plane is 10 x 18 voxels x 3 planes x CIC channels; its group planes, plane
// fastest, are one box plane apart, so one instruction's M rows (8 per group plane) cover the three
// z taps of CIC input channels: M = 64 for 16 channels (48 rows used), 128 for 32 (96 rows).  A
// block owns a chunk of CIC input channels and a slice of NCO output channels; for each 8 x 16 tile
// plane of its share of the work it receives, by two tensor copies, that input box and the
// gradient's 8 x 16 tile (the slice's groups), and one thread issues, per K step of 16 voxels (two
// tile rows), one instruction per (y, x) tap whose A start address is the box shifted by the tap.
// The nine accumulators stay in tensor memory (9 NCO FP32 columns) over all of the block's tiles;
// four warps add them to the FP32 gradient once at the end.  The M rows past the used ones read
// other shared memory and are not used.
//
// With M = 64 and 16 output channels (the finest layers) the x taps go into N as well: the
// gradient tile is received 10 voxels wide, and one instruction's N = 24 columns are its 8 channels
// of one group at three one-voxel shifts j = 0, 1, 2 (stride byte offset 16: the three core
// matrices overlap), paired with the input box at x offset 2, so that column group j holds x tap
// 2 - j; per K step that is 3 y taps x 2 groups = 6 instructions instead of 9.  Each shift sums the
// gradient over its tile's 8 voxels moved by j, so the tiles start one tile further left (x0 =
// -8, ...) to count every gradient voxel once at every shift.
template <int CIC, int NCO, int M>
struct WgCfg {
    static_assert((CIC == 16 && M == 64) || (CIC == 32 && M == 128), "input-channel chunk and rows");
    static_assert(NCO % 16 == 0, "output-channel slice");
    static constexpr bool XN = M == 64 && NCO == 16;                     // x taps in N
    static constexpr int DW = XN ? kBoxX : kTileX;                       // gradient box width
    static constexpr int XG = 3 * CIC / 8;                               // group planes of a box
    static constexpr int MG = M / 8, DG = NCO / 8;
    static constexpr int R = 4;                                          // ring slots
    static constexpr uint32_t XSLOT = (uint32_t)XG * kGroupBytes;        // input box (3 planes, halo)
    static constexpr uint32_t DGB = DW * kTileY * 16;                    // one gradient group
    static constexpr uint32_t DSLOT = (uint32_t)DG * DGB;
    static constexpr uint32_t TCOLS = pow2_at_least(9u * NCO);
    static constexpr size_t oX = 0;
    // the unused rows of the last slot read up to (MG - XG) group planes further on
    static constexpr size_t oD = al128((size_t)R * XSLOT + (size_t)(MG - XG) * kGroupBytes);
    static constexpr size_t oBar = oD + al128((size_t)R * DSLOT);
    static constexpr size_t SMEM_USED = al128(oBar + 8 * (2 * R + 1) + 8) + 128;   // + alignment slack
    // no more blocks per SM than tensor memory holds (512 columns per SM)
    static constexpr size_t SMEM = TCOLS == 512 ? (SMEM_USED > 120 * 1024 ? SMEM_USED : 120 * 1024)
                                 : TCOLS == 256 ? (SMEM_USED > 80 * 1024 ? SMEM_USED : 80 * 1024) : SMEM_USED;
    static_assert(SMEM <= 232448, "shared memory per block");
    static_assert(TCOLS <= 512, "tensor memory");
};

struct WgArgs {
    int tiles_x, tiles_y;     // tile columns along x (one more, starting at x0 = -8, with x taps in N)
    int x_first;              // x of the first tile column: 0, or -8 with x taps in N
    long long items;          // tile planes: tiles_x tiles_y nz
    long long per;            // tile planes per block
    int nchunks, nslices;     // input-channel chunks of CIC, output-channel slices of NCO
    int cin, cout;
    float* gw;                // [27][cout][cin], added to
    int* err;                 // set to 1 when a bounded wait runs out
};

// Block order: input-channel chunk fastest, then output slice, then the block's range of tile
// planes (the chunks and slices of a range read the same gradient and input tiles at nearly the
// same time, through L2).
template <int CIC, int NCO, int M>
__global__ void __launch_bounds__(kConvThreads, 1)
k_conv3_wgrad_umma(const __grid_constant__ CUtensorMap x_map, const __grid_constant__ CUtensorMap dy_map,
                   const WgArgs a) {
    using G = WgCfg<CIC, NCO, M>;
    constexpr int R = G::R;
    extern __shared__ unsigned char smraw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 127) & ~uintptr_t(127));
    unsigned char* xs = sm + G::oX;
    unsigned char* ds = sm + G::oD;
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + G::oBar);
    uint64_t* empty = full + R;
    uint64_t* done = empty + R;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int b = blockIdx.x;
    const int chunk = b % a.nchunks;
    b /= a.nchunks;
    const int slice = b % a.nslices;
    const long long blk = b / a.nslices;
    const long long it0 = blk * a.per;
    const int nitems = (int)max(0LL, min(a.items, it0 + a.per) - it0);
    const int ntiles = a.tiles_x * a.tiles_y;
    if (tid == 0) {
        for (int i = 0; i < R; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        mbar_init(done, 1);
        fence_mbar_init();
    }
    if (warp == 0) umma::tmem_alloc(tslot, G::TCOLS);
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = *tslot;
    bool fail = false;

    if (warp == 0) {
        if (lane == 0) {
            int issued = 0;
            for (int i = 0; i < nitems; ++i) {
                const int s = i % R;
                if (i >= R && !mbar_wait_bounded(&empty[s], (uint32_t)((i / R) - 1) & 1u)) {
                    fail = true;
                    break;
                }
                const long long item = it0 + i;
                const int tile = (int)(item % ntiles), z = (int)(item / ntiles);
                const int x0 = a.x_first + (tile % a.tiles_x) * kTileX, y0 = (tile / a.tiles_x) * kTileY;
                mbar_expect_tx(&full[s], G::XSLOT + G::DSLOT);
                umma::tma_load_5d(xs + (size_t)s * G::XSLOT, &x_map, &full[s], 0, x0 - 1, y0 - 1, z - 1, chunk * (CIC / 8));
                umma::tma_load_5d(ds + (size_t)s * G::DSLOT, &dy_map, &full[s], 0, x0, y0, z, slice * G::DG);
                ++issued;
            }
            // every copy issued must have landed before the block may leave
            for (int i = max(0, issued - R); i < issued; ++i)
                if (!mbar_wait_bounded(&full[i % R], (uint32_t)(i / R) & 1u)) fail = true;
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t id = G::XN ? umma::idesc_bf16_mn(M, 24) : umma::idesc_bf16_mn(M, NCO);
            const uint32_t xbase = umma::saddr(xs), dbase = umma::saddr(ds);
            for (int i = 0; i < nitems && !fail; ++i) {
                const int s = i % R;
                if (!mbar_wait_bounded(&full[s], (uint32_t)(i / R) & 1u)) {
                    fail = true;
                    break;
                }
                umma::fence_after_sync();
                const uint32_t xslot = xbase + (uint32_t)s * G::XSLOT, dslot = dbase + (uint32_t)s * G::DSLOT;
                // K steps outermost: consecutive instructions go to the nine taps' separate
                // accumulators
#pragma unroll 1
                for (int ks = 0; ks < kTileY / 2 && G::XN; ++ks) {
                    // K = tile rows 2 ks and 2 ks + 1: gradient box rows one box row (10 voxels)
                    // apart, the three shifts 16 bytes apart; input box at x offset 2, shifted by
                    // the y tap
#pragma unroll
                    for (int ty = 0; ty < 3; ++ty) {
                        const uint64_t ad =
                            umma::smem_desc(xslot + (uint32_t)(((2 * ks + ty) * kBoxX + 2) * 16), kBoxX * 16, kGroupBytes);
#pragma unroll
                        for (int cg = 0; cg < G::DG; ++cg) {
                            const uint64_t bd =
                                umma::smem_desc(dslot + (uint32_t)(cg * G::DGB + ks * 2 * G::DW * 16), G::DW * 16, 16);
                            umma::mma_bf16(tmem + (uint32_t)((ty * G::DG + cg) * 24), ad, bd, id,
                                           (i > 0 || ks > 0) ? 1u : 0u);
                        }
                    }
                }
#pragma unroll 1
                for (int ks = 0; ks < kTileY / 2 && !G::XN; ++ks) {
                    // K = tile rows 2 ks and 2 ks + 1 (8 voxels each): gradient tile rows one tile row
                    // apart, channel groups one group plane apart
                    const uint64_t bd = umma::smem_desc(dslot + (uint32_t)(ks * 2 * kTileX * 16), kTileX * 16, G::DGB);
#pragma unroll
                    for (int t = 0; t < 9; ++t) {
                        const int ty = t / 3, tx = t % 3;
                        // input box rows shifted by the tap, one box row (kBoxX voxels) apart; M
                        // groups (plane, channel group) one box plane apart
                        const uint64_t ad =
                            umma::smem_desc(xslot + (uint32_t)(((2 * ks + ty) * kBoxX + tx) * 16), kBoxX * 16, kGroupBytes);
                        umma::mma_bf16(tmem + (uint32_t)(t * NCO), ad, bd, id, (i > 0 || ks > 0) ? 1u : 0u);
                    }
                }
                umma::commit(&empty[s]);   // the slot may be refilled
            }
            umma::commit(done);            // every MMA issued has completed
        }
    } else {
        // epilogue: warp quarter q of the TMEM lanes; accumulator row of this lane (M = 64: the
        // first 16 lanes of each quarter), its group plane m (channel group m / 3, z tap m % 3)
        const int q = warp & 3;
        const int row = M == 128 ? q * 32 + lane : (lane < 16 ? q * 16 + lane : M);
        const int m = row >> 3;
        const bool used = row < M && m < G::XG;
        const int ci = chunk * CIC + (m / 3) * 8 + (row & 7), tz = m % 3;
        if (!mbar_wait_bounded(done, 0u)) fail = true;
        if (!__any_sync(0xffffffffu, fail) && nitems > 0) {
            umma::fence_after_sync();
#pragma unroll 1
            for (int c0 = 0; c0 < 9 * NCO; c0 += 16) {
                uint32_t r[16];
                umma::tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, r);
                umma::tmem_wait_ld();
                if (used) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        // column c: (y tap, group, shift, channel) with x taps in N, else (tap, channel)
                        const int c = c0 + j;
                        int tap, co;
                        if constexpr (G::XN) {
                            const int blk = c / 24, rem = c % 24;
                            tap = 9 * tz + 3 * (blk / G::DG) + (2 - rem / 8);
                            co = 8 * (blk % G::DG) + (rem & 7);
                        } else {
                            tap = 9 * tz + c / NCO;
                            co = c % NCO;
                        }
                        atomicAdd(a.gw + ((long long)tap * a.cout + slice * NCO + co) * a.cin + ci, __uint_as_float(r[j]));
                    }
                }
            }
        }
    }
    if (fail) atomicExch(a.err, 1);
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        umma::fence_after_sync();
        umma::tmem_dealloc(tmem, G::TCOLS);
    }
}

// ---- small kernels (chunk-planar tensors) ---------------------------------------------------------
// dpre = dy where y > 0 (ReLU gradient), in place on dy (same layout and channel count)
__global__ void k_relu_bwd(bf16* __restrict__ dy, const bf16* __restrict__ y, long long n) {
    const bf16 zero = __float2bfloat16(0.f);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        if (!(__bfloat162float(y[i]) > 0.f)) dy[i] = zero;
}

__device__ __forceinline__ void unpack8(const uint4& u, float (&f)[8]) {
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        f[2 * h] = __uint_as_float(w[h] << 16);
        f[2 * h + 1] = __uint_as_float(w[h] & 0xFFFF0000u);
    }
}
// db[8 g + j] += sum over voxels of dy[v][8 g + j] (channel group g = blockIdx.y): one 16-byte
// word (the group's 8 channels of a voxel) per thread and voxel, eight sums per thread, reduced
// over the warp by shuffles and over the block in shared memory
__global__ void __launch_bounds__(256) k_bias_grad(const bf16* __restrict__ dy, long long nv, float* __restrict__ db) {
    __shared__ float sh[8][8];
    const int g = blockIdx.y;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const uint4* src = reinterpret_cast<const uint4*>(dy) + (long long)g * nv;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nv; v += (long long)gridDim.x * blockDim.x) {
        float f[8];
        unpack8(src[v], f);
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j] += f[j];
    }
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
#pragma unroll
        for (int j = 0; j < 8; ++j) sh[warp][j] = acc[j];
    __syncthreads();
    if (threadIdx.x < 8) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w][threadIdx.x];
        atomicAdd(db + 8 * g + threadIdx.x, t);
    }
}

__device__ __forceinline__ uint4 pack8(const float (&f)[8]) {
    uint32_t w[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        const __nv_bfloat162 p = __floats2bfloat162_rn(f[2 * h], f[2 * h + 1]);
        w[h] = *reinterpret_cast<const uint32_t*>(&p);
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}
__device__ __forceinline__ long long parent_voxel(long long v, int nx, int ny) {
    const int x = int(v % nx), y = int((v / nx) % ny);
    const long long z = v / ((long long)nx * ny);
    return ((z / 2) * (ny / 2) + y / 2) * (nx / 2) + x / 2;
}

// 2x2x2 average pooling of `groups` channel groups: (nx,ny,nz) -> (nx/2,ny/2,nz/2)
__global__ void k_pool(const bf16* __restrict__ in, bf16* __restrict__ out, int nx, int ny, int nz, int groups) {
    const int hx = nx / 2, hy = ny / 2, hz = nz / 2;
    const long long Vf = (long long)nx * ny * nz, Vc = (long long)hx * hy * hz;
    const uint4* src = reinterpret_cast<const uint4*>(in);
    uint4* dst = reinterpret_cast<uint4*>(out);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < Vc * groups; i += (long long)gridDim.x * blockDim.x) {
        const int k = int(i / Vc);
        const long long v = i % Vc;
        const int x = int(v % hx), y = int((v / hx) % hy), z = int(v / ((long long)hx * hy));
        float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int q = 0; q < 8; ++q) {
            const int xx = 2 * x + (q & 1), yy = 2 * y + ((q >> 1) & 1), zz = 2 * z + (q >> 2);
            float f[8];
            unpack8(src[k * Vf + ((long long)zz * ny + yy) * nx + xx], f);
#pragma unroll
            for (int e = 0; e < 8; ++e) s[e] += f[e];
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) s[e] *= 0.125f;
        dst[k * Vc + v] = pack8(s);
    }
}

// gradient of the pooling, added into din (din += dout(parent) / 8), `groups` channel groups
__global__ void k_pool_bwd(const bf16* __restrict__ dout, bf16* __restrict__ din, int nx, int ny, int nz, int groups,
                           int accumulate) {
    const long long Vf = (long long)nx * ny * nz, Vc = Vf / 8;
    const uint4* src = reinterpret_cast<const uint4*>(dout);
    uint4* dst = reinterpret_cast<uint4*>(din);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < Vf * groups; i += (long long)gridDim.x * blockDim.x) {
        const int k = int(i / Vf);
        const long long v = i % Vf;
        float g[8], d[8];
        unpack8(src[k * Vc + parent_voxel(v, nx, ny)], g);
        if (accumulate) unpack8(dst[i], d);
#pragma unroll
        for (int e = 0; e < 8; ++e) d[e] = accumulate ? d[e] + 0.125f * g[e] : 0.125f * g[e];
        dst[i] = pack8(d);
    }
}

// nearest upsampling of `groups` coarse channel groups into the first groups of a fine tensor
__global__ void k_upsample(const bf16* __restrict__ coarse, bf16* __restrict__ fine, int nx, int ny, int nz, int groups) {
    const long long Vf = (long long)nx * ny * nz, Vc = Vf / 8;
    const uint4* src = reinterpret_cast<const uint4*>(coarse);
    uint4* dst = reinterpret_cast<uint4*>(fine);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < Vf * groups; i += (long long)gridDim.x * blockDim.x) {
        const int k = int(i / Vf);
        dst[i] = src[k * Vc + parent_voxel(i % Vf, nx, ny)];
    }
}

// gradient of the upsampling: coarse (groups) = sum over each voxel's 8 children (fine groups 0..)
__global__ void k_upsample_bwd(const bf16* __restrict__ dfine, bf16* __restrict__ dcoarse, int nx, int ny, int nz,
                               int groups) {
    const int hx = nx / 2, hy = ny / 2, hz = nz / 2;
    const long long Vf = (long long)nx * ny * nz, Vc = (long long)hx * hy * hz;
    const uint4* src = reinterpret_cast<const uint4*>(dfine);
    uint4* dst = reinterpret_cast<uint4*>(dcoarse);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < Vc * groups; i += (long long)gridDim.x * blockDim.x) {
        const int k = int(i / Vc);
        const long long v = i % Vc;
        const int x = int(v % hx), y = int((v / hx) % hy), z = int(v / ((long long)hx * hy));
        float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int q = 0; q < 8; ++q) {
            const int xx = 2 * x + (q & 1), yy = 2 * y + ((q >> 1) & 1), zz = 2 * z + (q >> 2);
            float f[8];
            unpack8(src[k * Vf + ((long long)zz * ny + yy) * nx + xx], f);
#pragma unroll
            for (int e = 0; e < 8; ++e) s[e] += f[e];
        }
        dst[i] = pack8(s);
    }
}

// dst (+)= src over n 8-channel records (the skip branch of a concatenation's gradient)
__global__ void k_add_groups(const bf16* __restrict__ src, bf16* __restrict__ dst, long long nrec, int accumulate) {
    const uint4* s4 = reinterpret_cast<const uint4*>(src);
    uint4* d4 = reinterpret_cast<uint4*>(dst);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nrec; i += (long long)gridDim.x * blockDim.x) {
        if (!accumulate) {
            d4[i] = s4[i];
            continue;
        }
        float a[8], b[8];
        unpack8(s4[i], a);
        unpack8(d4[i], b);
#pragma unroll
        for (int e = 0; e < 8; ++e) b[e] += a[e];
        d4[i] = pack8(b);
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
    int nout_f, nout_b;      // output channels per block of the forward / data-gradient convolution
    float *w = nullptr, *b = nullptr, *gw = nullptr, *gb = nullptr;
    float *mw = nullptr, *vw = nullptr, *mb = nullptr, *vb = nullptr;
    bf16 *blob_f = nullptr, *blob_b = nullptr;
    long long nw() const { return 27LL * cout * cin; }
};

// encoder 1, 2, 3, decoder 2, 1 (two 3x3x3 convolutions each): stored input channels, output
// channels, real input channels, output channels per block forward and for the data gradient
// (the widest ones split so that weights and input ring fit one block's shared memory)
const int kLayers[10][5] = {{16, 16, 8, 16, 16},  {16, 16, 16, 16, 16}, {16, 32, 16, 32, 16}, {32, 32, 32, 32, 32},
                            {32, 64, 32, 64, 32}, {64, 64, 64, 32, 32}, {96, 32, 96, 16, 48}, {32, 32, 32, 32, 32},
                            {48, 16, 48, 16, 48}, {16, 16, 16, 16, 16}};

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
    int* derr = nullptr;      // device flag of the convolutions' bounded waits
    // grid-dependent
    int nx = 0, ny = 0, nz = 0;
    long long V1 = 0, V2 = 0, V3 = 0;
    std::vector<void*> grid_allocs, grad_allocs;
    // forward activations; s1 and s2 live in the last groups of the concatenations c1 and c2
    bf16 *geo = nullptr, *x0 = nullptr, *a1 = nullptr, *c1 = nullptr, *p1 = nullptr, *a2 = nullptr, *c2 = nullptr;
    bf16 *p2 = nullptr, *a3 = nullptr, *b3 = nullptr, *d2a = nullptr, *d2b = nullptr, *d1a = nullptr, *d1b = nullptr;
    bf16 *s1 = nullptr, *s2 = nullptr;
    // gradients (allocated by the first training step)
    bf16 *g16a = nullptr, *g16b = nullptr, *g48 = nullptr, *g32a = nullptr, *g32b = nullptr, *g96 = nullptr;
    bf16 *g64a = nullptr, *g64b = nullptr, *gs1 = nullptr, *gs2 = nullptr, *gp1 = nullptr, *gp2 = nullptr;
    float *mask = nullptr, *out = nullptr, *scal = nullptr;   // scal: sum r^2, count, scale, inv scale, loss
    bool bound = false, grads_ready = false;
    std::map<std::tuple<const void*, int, int, int, int>, CUtensorMap> maps;
    // other boxes: (tensor, nx, ny, nz, groups, box x y z, box groups)
    std::map<std::tuple<const void*, int, int, int, int, int, int>, CUtensorMap> tile_maps;

    template <typename T>
    vofp_status alloc(T** p, size_t count, std::vector<void*>& list) {
        void* q = nullptr;
        if (cudaMalloc(&q, sizeof(T) * (count ? count : 1)) != cudaSuccess) {
            err = "cudaMalloc failed";
            return VOFP_ERR_OOM;
        }
        list.push_back(q);
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
// first channel group of the input: the seven geometry channels and the residual over its RMS
// (the second group stays zero)
__global__ void k_pack_input_dev(const bf16* __restrict__ geo, const float* __restrict__ r, const float* scal,
                                 bf16* __restrict__ x, long long nv) {
    const float inv = scal[3];
    const uint4* g4 = reinterpret_cast<const uint4*>(geo);
    uint4* x4 = reinterpret_cast<uint4*>(x);
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nv; v += (long long)gridDim.x * blockDim.x) {
        uint4 u = g4[v];
        const __nv_bfloat16 rb = __float2bfloat16(r[v] * inv);
        u.w = (u.w & 0x0000FFFFu) | ((uint32_t)__bfloat16_as_ushort(rb) << 16);
        x4[v] = u;
    }
}
__global__ void k_head_dev(const bf16* __restrict__ h, const float* __restrict__ w, const float* __restrict__ b,
                           const float* scal, const float* __restrict__ mask, float* __restrict__ out, long long nv) {
    const float scale = scal[2];
    const uint4* h4 = reinterpret_cast<const uint4*>(h);
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nv; v += (long long)gridDim.x * blockDim.x) {
        float f0[8], f1[8];
        unpack8(h4[v], f0);
        unpack8(h4[nv + v], f1);
        float s = b[0];
#pragma unroll
        for (int c = 0; c < 8; ++c) s = fmaf(w[c], f0[c], s);
#pragma unroll
        for (int c = 0; c < 8; ++c) s = fmaf(w[8 + c], f1[c], s);
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
    const uint4* h4 = reinterpret_cast<const uint4*>(h);
    uint4* d4 = reinterpret_cast<uint4*>(dh);
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nv; v += (long long)gridDim.x * blockDim.x) {
        const float e = mask[v] * (out[v] - target[v]) * inv_scale;
        ll += e * e;
        const float go = 2.f * e * inv_count;
        lb += go;
        float f[2][8], g[2][8];
        unpack8(h4[v], f[0]);
        unpack8(h4[nv + v], f[1]);
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            lw[c] = fmaf(go, f[c >> 3][c & 7], lw[c]);
            g[c >> 3][c & 7] = go * w[c];
        }
        d4[v] = pack8(g[0]);
        d4[nv + v] = pack8(g[1]);
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

// output layer's backward pass from a given gradient dL/dz of the network output z
// (z = mask (b + w . h) scale): dL/ds = dz mask scale per voxel
__global__ void k_head_bwd_given(const bf16* __restrict__ h, const float* __restrict__ w, const float* __restrict__ dz,
                                 const float* __restrict__ mask, const float* scal, bf16* __restrict__ dh,
                                 float* __restrict__ dw, float* __restrict__ db, long long nv) {
    __shared__ float sh[17][128];
    const float scale = scal[2];
    float lw[16], lb = 0.f;
#pragma unroll
    for (int c = 0; c < 16; ++c) lw[c] = 0.f;
    const uint4* h4 = reinterpret_cast<const uint4*>(h);
    uint4* d4 = reinterpret_cast<uint4*>(dh);
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nv; v += (long long)gridDim.x * blockDim.x) {
        const float go = dz[v] * mask[v] * scale;
        lb += go;
        float f[2][8], g[2][8];
        unpack8(h4[v], f[0]);
        unpack8(h4[nv + v], f[1]);
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            lw[c] = fmaf(go, f[c >> 3][c & 7], lw[c]);
            g[c >> 3][c & 7] = go * w[c];
        }
        d4[v] = pack8(g[0]);
        d4[nv + v] = pack8(g[1]);
    }
#pragma unroll
    for (int c = 0; c < 16; ++c) sh[c][threadIdx.x] = lw[c];
    sh[16][threadIdx.x] = lb;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int c = 0; c < 17; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x < 16) atomicAdd(dw + threadIdx.x, sh[threadIdx.x][0]);
    if (threadIdx.x == 16) atomicAdd(db, sh[16][0]);
}

// chunk-planar tensor map: five dimensions (8 channels, x, y, z, channel group), box of one
// halo'd 10 x 18 tile plane of every group (cached per tensor and level)
const CUtensorMap* act_map(vofp_nn* n, const bf16* ptr, int nx, int ny, int nz, int groups) {
    const auto key = std::make_tuple((const void*)ptr, nx, ny, nz, groups);
    auto it = n->maps.find(key);
    if (it != n->maps.end()) return &it->second;
    auto enc = tensor_map_encoder();
    if (!enc) return nullptr;
    CUtensorMap m;
    std::memset(&m, 0, sizeof(m));
    const cuuint64_t V = (cuuint64_t)nx * ny * nz;
    const cuuint64_t dims[5] = {8, (cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz, (cuuint64_t)groups};
    const cuuint64_t strides[4] = {16, (cuuint64_t)nx * 16, (cuuint64_t)nx * ny * 16, V * 16};
    const cuuint32_t box[5] = {8, (cuuint32_t)kBoxX, (cuuint32_t)kBoxY, 1, (cuuint32_t)groups};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    const CUresult r = enc(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<bf16*>(ptr), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return nullptr;
    return &(n->maps[key] = m);
}

// chunk-planar tensor map with a box of bx x by voxels, bz planes and box_groups channel groups
// (cached per tensor, level and box)
const CUtensorMap* box_map(vofp_nn* n, const bf16* ptr, int nx, int ny, int nz, int groups, int bx, int by, int bz,
                           int box_groups) {
    const auto key = std::make_tuple((const void*)ptr, nx, ny, nz, groups, bx * 1000000 + by * 1000 + bz, box_groups);
    auto it = n->tile_maps.find(key);
    if (it != n->tile_maps.end()) return &it->second;
    auto enc = tensor_map_encoder();
    if (!enc) return nullptr;
    CUtensorMap m;
    std::memset(&m, 0, sizeof(m));
    const cuuint64_t V = (cuuint64_t)nx * ny * nz;
    const cuuint64_t dims[5] = {8, (cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz, (cuuint64_t)groups};
    const cuuint64_t strides[4] = {16, (cuuint64_t)nx * 16, (cuuint64_t)nx * ny * 16, V * 16};
    const cuuint32_t box[5] = {8, (cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz, (cuuint32_t)box_groups};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    const CUresult r = enc(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<bf16*>(ptr), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return nullptr;
    return &(n->tile_maps[key] = m);
}

template <int CIC, int NCO, int M>
vofp_status wgrad_umma(vofp_nn* n, const CUtensorMap* xm, const CUtensorMap* dm, WgArgs a) {
    using G = WgCfg<CIC, NCO, M>;
    auto kern = k_conv3_wgrad_umma<CIC, NCO, M>;
    static int occ = -1;   // resident blocks per SM (per instantiation; one device per process)
    if (occ < 0) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kConvThreads, G::SMEM) != cudaSuccess || occ < 1) {
            occ = -1;
            n->err = "tensor-core weight gradient: shared memory opt-in failed";
            return VOFP_ERR_CUDA;
        }
    }
    // one wave: the resident blocks shared by the chunks and slices, each block a run of at least
    // four tile planes
    const long long groups = (long long)a.nchunks * a.nslices;
    const long long want = std::max(1LL, (long long)num_sms() * occ / groups);
    a.per = std::max(4LL, (a.items + want - 1) / want);
    const long long nb = (a.items + a.per - 1) / a.per;
    a.err = n->derr;
    kern<<<(unsigned)(nb * groups), kConvThreads, G::SMEM, n->stream>>>(*xm, *dm, a);
    return cudaGetLastError() == cudaSuccess ? VOFP_OK : VOFP_ERR_CUDA;
}

template <int CIN, int NOUT, int R>
vofp_status conv_umma(vofp_nn* n, const CUtensorMap* map, ConvArgs a, int nsplit) {
    using G = ConvCfg<CIN, NOUT, R>;
    auto kern = k_conv3_umma<CIN, NOUT, R>;
    static int occ = -1;   // resident blocks per SM (per instantiation; one device per process)
    if (occ < 0) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kConvThreads, G::SMEM) != cudaSuccess || occ < 1) {
            occ = -1;
            n->err = "tensor-core convolution: shared memory opt-in failed";
            return VOFP_ERR_CUDA;
        }
    }
    // z segments of at most S planes (the accumulators one block keeps in tensor memory), equal
    // in length; each re-reads a 2-plane halo
    const long long cols = (long long)a.tiles_x * a.tiles_y * nsplit;
    const int nseg = (a.nz + G::S - 1) / G::S;
    a.seg = (a.nz + nseg - 1) / nseg;
    a.nseg = (a.nz + a.seg - 1) / a.seg;
    a.err = n->derr;
    const long long blocks = cols * a.nseg;
    kern<<<(unsigned)blocks, kConvThreads, G::SMEM, n->stream>>>(*map, a);
    return cudaGetLastError() == cudaSuccess ? VOFP_OK : VOFP_ERR_CUDA;
}

// One 3x3x3 convolution of `in` (cin channels) into groups [out_chunk0, ...) of `out` (cout
// channels in blocks of nout): the layer's forward weights, or its data-gradient weights (taps
// mirrored, channels transposed; no bias, no ReLU).
vofp_status conv(vofp_nn* n, const bf16* in, int cin, const bf16* blob, int cout, int nout, const float* bias,
                 bool relu, bf16* out, int out_chunk0, int nx, int ny, int nz) {
    const CUtensorMap* map = act_map(n, in, nx, ny, nz, cin / 8);
    if (!map) {
        n->err = "tensor map of an activation could not be built";
        return VOFP_ERR_CUDA;
    }
    ConvArgs a{};
    a.nx = nx;
    a.ny = ny;
    a.nz = nz;
    a.tiles_x = (nx + kTileX - 1) / kTileX;
    a.tiles_y = (ny + kTileY - 1) / kTileY;
    a.V = (long long)nx * ny * nz;
    a.bias = bias;
    a.relu = relu ? 1 : 0;
    a.wblob = blob;
    a.out = out;
    a.out_chunk0 = out_chunk0;
    const int ns = cout / nout;
    switch (cin * 1000 + nout) {
        case 16016: return conv_umma<16, 16, 4>(n, map, a, ns);
        case 16032: return conv_umma<16, 32, 4>(n, map, a, ns);
        case 16048: return conv_umma<16, 48, 4>(n, map, a, ns);
        case 32016: return conv_umma<32, 16, 4>(n, map, a, ns);
        case 32032: return conv_umma<32, 32, 4>(n, map, a, ns);
        case 32048: return conv_umma<32, 48, 4>(n, map, a, ns);
        case 32064: return conv_umma<32, 64, 4>(n, map, a, ns);
        case 48016: return conv_umma<48, 16, 4>(n, map, a, ns);
        case 64032: return conv_umma<64, 32, 4>(n, map, a, ns);
        case 96016: return conv_umma<96, 16, 4>(n, map, a, ns);
        default: n->err = "no tensor-core convolution for this shape"; return VOFP_ERR_INVALID_ARG;
    }
}

vofp_status conv_fwd(vofp_nn* n, const Layer& l, const bf16* in, bf16* out, int out_chunk0, int nx, int ny, int nz) {
    return conv(n, in, l.cin, l.blob_f, l.cout, l.nout_f, l.b, true, out, out_chunk0, nx, ny, nz);
}

// weight and bias gradients of one layer from its input x and the gradient dy of its output
// (before the ReLU), added to l.gw and l.gb
vofp_status conv_wgrad(vofp_nn* n, const bf16* x, const bf16* dy, const Layer& l, int nx, int ny, int nz) {
    const int nco = l.cout == 16 ? 16 : 32;
    const int cic = l.cin % 32 == 0 ? 32 : 16;
    const CUtensorMap* xm = box_map(n, x, nx, ny, nz, l.cin / 8, kBoxX, kBoxY, 3, cic / 8);
    const bool xn = cic == 16 && nco == 16;   // x taps in N (WgCfg::XN): 10-voxel gradient box
    const CUtensorMap* dm = box_map(n, dy, nx, ny, nz, l.cout / 8, xn ? kBoxX : kTileX, kTileY, 1, nco / 8);
    if (!xm || !dm) {
        n->err = "tensor map of an activation could not be built";
        return VOFP_ERR_CUDA;
    }
    WgArgs a{};
    a.tiles_x = (nx + kTileX - 1) / kTileX + (xn ? 1 : 0);
    a.x_first = xn ? -kTileX : 0;
    a.tiles_y = (ny + kTileY - 1) / kTileY;
    a.items = (long long)a.tiles_x * a.tiles_y * nz;
    a.nchunks = l.cin / cic;
    a.nslices = l.cout / nco;
    a.cin = l.cin;
    a.cout = l.cout;
    a.gw = l.gw;
    vofp_status s;
    switch (cic * 1000 + nco) {
        case 16016: s = wgrad_umma<16, 16, 64>(n, xm, dm, a); break;
        case 16032: s = wgrad_umma<16, 32, 64>(n, xm, dm, a); break;
        case 32032: s = wgrad_umma<32, 32, 128>(n, xm, dm, a); break;
        default: n->err = "no tensor-core weight gradient for this shape"; return VOFP_ERR_INVALID_ARG;
    }
    if (s) return s;
    const long long nv = (long long)nx * ny * nz;
    const int bx = (int)std::max(1LL, std::min((long long)num_sms() * 8 / (l.cout / 8), (nv + 255) / 256));
    k_bias_grad<<<dim3(bx, l.cout / 8), 256, 0, n->stream>>>(dy, nv, l.gb);
    return VOFP_OK;
}

void refresh_blobs(vofp_nn* n) {
    for (auto& l : n->L) {
        k_blob_fwd<<<gs(l.nw()), 256, 0, n->stream>>>(l.w, l.cout, l.cin, l.nout_f, l.blob_f);
        k_blob_dgrad<<<gs(l.nw()), 256, 0, n->stream>>>(l.w, l.cout, l.cin, l.nout_b, l.blob_b);
    }
}

vofp_status check_err(vofp_nn* n) {
    if (cudaGetLastError() != cudaSuccess) {
        n->err = "kernel launch failed";
        return VOFP_ERR_CUDA;
    }
    return VOFP_OK;
}

// forward pass on stream st (the network's own stream unless a caller orders it elsewhere)
vofp_status forward(vofp_nn* n, const float* r) {
    cudaStream_t st = n->stream;
    const int X = n->nx, Y = n->ny, Z = n->nz;
    const int X2 = X / 2, Y2 = Y / 2, Z2 = Z / 2, X4 = X / 4, Y4 = Y / 4, Z4 = Z / 4;
    cudaMemsetAsync(n->scal, 0, sizeof(float) * 8, st);
    k_rms<<<gs(n->V1), 256, 0, st>>>(r, n->mask, n->V1, n->scal);
    k_rms_finish<<<1, 1, 0, st>>>(n->scal);
    k_pack_input_dev<<<gs(n->V1), 256, 0, st>>>(n->geo, r, n->scal, n->x0, n->V1);
    auto& L = n->L;
    vofp_status s;
    if ((s = conv_fwd(n, L[0], n->x0, n->a1, 0, X, Y, Z)) || (s = conv_fwd(n, L[1], n->a1, n->c1, 4, X, Y, Z)))
        return s;
    k_pool<<<gs(n->V2 * 2), 256, 0, st>>>(n->s1, n->p1, X, Y, Z, 2);
    if ((s = conv_fwd(n, L[2], n->p1, n->a2, 0, X2, Y2, Z2)) || (s = conv_fwd(n, L[3], n->a2, n->c2, 8, X2, Y2, Z2)))
        return s;
    k_pool<<<gs(n->V3 * 4), 256, 0, st>>>(n->s2, n->p2, X2, Y2, Z2, 4);
    if ((s = conv_fwd(n, L[4], n->p2, n->a3, 0, X4, Y4, Z4)) || (s = conv_fwd(n, L[5], n->a3, n->b3, 0, X4, Y4, Z4)))
        return s;
    k_upsample<<<gs(n->V2 * 8), 256, 0, st>>>(n->b3, n->c2, X2, Y2, Z2, 8);
    if ((s = conv_fwd(n, L[6], n->c2, n->d2a, 0, X2, Y2, Z2)) || (s = conv_fwd(n, L[7], n->d2a, n->d2b, 0, X2, Y2, Z2)))
        return s;
    k_upsample<<<gs(n->V1 * 4), 256, 0, st>>>(n->d2b, n->c1, X, Y, Z, 4);
    if ((s = conv_fwd(n, L[8], n->c1, n->d1a, 0, X, Y, Z)) || (s = conv_fwd(n, L[9], n->d1a, n->d1b, 0, X, Y, Z)))
        return s;
    k_head_dev<<<gs(n->V1), 256, 0, st>>>(n->d1b, n->hw, n->hb, n->scal, n->mask, n->out, n->V1);
    return check_err(n);
}

// gradient of one conv layer y = relu(conv(x)): dy (BF16, in place -> dpre), weight/bias grads,
// and optionally the input gradient dx (data-gradient convolution on the tensor cores)
vofp_status layer_bwd(vofp_nn* n, const Layer& l, const bf16* x, const bf16* y, bf16* dy, bf16* dx, int nx, int ny,
                      int nz) {
    const long long nv = (long long)nx * ny * nz;
    k_relu_bwd<<<gs(nv * l.cout), 256, 0, n->stream>>>(dy, y, nv * l.cout);
    if (vofp_status s = conv_wgrad(n, x, dy, l, nx, ny, nz)) return s;
    if (dx) return conv(n, dy, l.cout, l.blob_b, l.cin, l.nout_b, nullptr, false, dx, 0, nx, ny, nz);
    return VOFP_OK;
}

// backward pass after forward(): from the mean-squared error against `target`, or from a given
// gradient dz of the output when target is null
vofp_status backward(vofp_nn* n, const float* target, const float* dz = nullptr) {
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
    if (target)
        k_head_bwd_dev<<<gs(n->V1, 128), 128, 0, st>>>(n->d1b, n->hw, n->out, target, n->mask, n->scal, n->g16a,
                                                       n->ghw, n->ghb, n->V1);
    else
        k_head_bwd_given<<<gs(n->V1, 128), 128, 0, st>>>(n->d1b, n->hw, dz, n->mask, n->scal, n->g16a, n->ghw, n->ghb,
                                                         n->V1);
    vofp_status s;
    if ((s = layer_bwd(n, L[9], n->d1a, n->d1b, n->g16a, n->g16b, X, Y, Z))) return s;   // -> d(d1a)
    if ((s = layer_bwd(n, L[8], n->c1, n->d1a, n->g16b, n->g48, X, Y, Z))) return s;     // -> d(c1)
    k_upsample_bwd<<<gs(n->V2 * 4), 256, 0, st>>>(n->g48, n->g32a, X, Y, Z, 4);          // -> d(d2b)
    k_add_groups<<<gs(n->V1 * 2), 256, 0, st>>>(n->g48 + 4 * n->V1 * 8, n->gs1, n->V1 * 2, 0);   // skip 1
    if ((s = layer_bwd(n, L[7], n->d2a, n->d2b, n->g32a, n->g32b, X2, Y2, Z2))) return s;  // -> d(d2a)
    if ((s = layer_bwd(n, L[6], n->c2, n->d2a, n->g32b, n->g96, X2, Y2, Z2))) return s;    // -> d(c2)
    k_upsample_bwd<<<gs(n->V3 * 8), 256, 0, st>>>(n->g96, n->g64a, X2, Y2, Z2, 8);        // -> d(b3)
    k_add_groups<<<gs(n->V2 * 4), 256, 0, st>>>(n->g96 + 8 * n->V2 * 8, n->gs2, n->V2 * 4, 0);   // skip 2
    if ((s = layer_bwd(n, L[5], n->a3, n->b3, n->g64a, n->g64b, X4, Y4, Z4))) return s;    // -> d(a3)
    if ((s = layer_bwd(n, L[4], n->p2, n->a3, n->g64b, n->gp2, X4, Y4, Z4))) return s;     // -> d(p2)
    k_pool_bwd<<<gs(n->V2 * 4), 256, 0, st>>>(n->gp2, n->gs2, X2, Y2, Z2, 4, 1);
    if ((s = layer_bwd(n, L[3], n->a2, n->s2, n->gs2, n->g32a, X2, Y2, Z2))) return s;     // -> d(a2)
    if ((s = layer_bwd(n, L[2], n->p1, n->a2, n->g32a, n->gp1, X2, Y2, Z2))) return s;     // -> d(p1)
    k_pool_bwd<<<gs(n->V1 * 2), 256, 0, st>>>(n->gp1, n->gs1, X, Y, Z, 2, 1);
    if ((s = layer_bwd(n, L[1], n->a1, n->s1, n->gs1, n->g16a, X, Y, Z))) return s;        // -> d(a1)
    if ((s = layer_bwd(n, L[0], n->x0, n->a1, n->g16a, nullptr, X, Y, Z))) return s;
    return check_err(n);
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
    refresh_blobs(n);
}

void free_list(std::vector<void*>& list) {
    for (void* p : list) cudaFree(p);
    list.clear();
}

vofp_status ensure_grid(vofp_nn* n, int nx, int ny, int nz) {
    if (nx % 4 || ny % 4 || nz % 4 || nx < 4 || ny < 4 || nz < 4) {
        n->err = "grid sizes must be positive multiples of 4 (two 2x2x2 poolings)";
        return VOFP_ERR_INVALID_ARG;
    }
    if (n->bound && n->nx == nx && n->ny == ny && n->nz == nz) return VOFP_OK;
    cudaStreamSynchronize(n->stream);
    free_list(n->grid_allocs);
    free_list(n->grad_allocs);
    n->maps.clear();
    n->tile_maps.clear();
    n->bound = false;
    n->grads_ready = false;
    n->nx = nx;
    n->ny = ny;
    n->nz = nz;
    n->V1 = (long long)nx * ny * nz;
    n->V2 = n->V1 / 8;
    n->V3 = n->V1 / 64;
    const long long V1 = n->V1, V2 = n->V2, V3 = n->V3;
    auto& g = n->grid_allocs;
    vofp_status s;
    if ((s = n->alloc(&n->geo, V1 * 8, g)) || (s = n->alloc(&n->x0, V1 * 16, g)) || (s = n->alloc(&n->a1, V1 * 16, g)) ||
        (s = n->alloc(&n->c1, V1 * 48, g)) || (s = n->alloc(&n->p1, V2 * 16, g)) || (s = n->alloc(&n->a2, V2 * 32, g)) ||
        (s = n->alloc(&n->c2, V2 * 96, g)) || (s = n->alloc(&n->p2, V3 * 32, g)) || (s = n->alloc(&n->a3, V3 * 64, g)) ||
        (s = n->alloc(&n->b3, V3 * 64, g)) || (s = n->alloc(&n->d2a, V2 * 32, g)) || (s = n->alloc(&n->d2b, V2 * 32, g)) ||
        (s = n->alloc(&n->d1a, V1 * 16, g)) || (s = n->alloc(&n->d1b, V1 * 16, g)) || (s = n->alloc(&n->mask, V1, g)) ||
        (s = n->alloc(&n->out, V1, g)))
        return s;
    n->s1 = n->c1 + 4 * V1 * 8;   // the skip tensors are the last groups of the concatenations
    n->s2 = n->c2 + 8 * V2 * 8;
    // the input's second channel group is always zero (seven geometry channels and the residual)
    if (cudaMemsetAsync(n->x0 + V1 * 8, 0, sizeof(bf16) * V1 * 8, n->stream) != cudaSuccess) return VOFP_ERR_CUDA;
    n->bound = true;
    return VOFP_OK;
}

vofp_status ensure_grads(vofp_nn* n) {
    if (n->grads_ready) return VOFP_OK;
    const long long V1 = n->V1, V2 = n->V2, V3 = n->V3;
    auto& g = n->grad_allocs;
    vofp_status s;
    if ((s = n->alloc(&n->g16a, V1 * 16, g)) || (s = n->alloc(&n->g16b, V1 * 16, g)) ||
        (s = n->alloc(&n->g48, V1 * 48, g)) || (s = n->alloc(&n->g32a, V2 * 32, g)) ||
        (s = n->alloc(&n->g32b, V2 * 32, g)) || (s = n->alloc(&n->g96, V2 * 96, g)) ||
        (s = n->alloc(&n->g64a, V3 * 64, g)) || (s = n->alloc(&n->g64b, V3 * 64, g)) ||
        (s = n->alloc(&n->gs1, V1 * 16, g)) || (s = n->alloc(&n->gs2, V2 * 32, g)) ||
        (s = n->alloc(&n->gp1, V2 * 16, g)) || (s = n->alloc(&n->gp2, V3 * 32, g)))
        return s;
    n->grads_ready = true;
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

// the convolutions' device flag: a bounded wait that ran out is an error of the whole pass
vofp_status read_err(vofp_nn* n) {
    int h = 0;
    if (cudaMemcpyAsync(&h, n->derr, sizeof(int), cudaMemcpyDeviceToHost, n->stream) != cudaSuccess ||
        cudaStreamSynchronize(n->stream) != cudaSuccess)
        return VOFP_ERR_CUDA;
    if (h) {
        n->err = "a tensor-core convolution's bounded wait ran out";
        cudaMemsetAsync(n->derr, 0, sizeof(int), n->stream);
        return VOFP_ERR_DEVICE_TIMEOUT;
    }
    return VOFP_OK;
}

}  // namespace
}  // namespace nn
}  // namespace vofp

using namespace vofp::nn;

namespace vofp {
namespace nn {
long long bound_cells(const vofp_nn* n) { return n && n->bound ? n->V1 : -1; }
cudaStream_t stream_of(const vofp_nn* n) { return n ? n->stream : nullptr; }
vofp_status forward_on(vofp_nn* n, cudaStream_t st, const float* r) {
    const cudaStream_t own = n->stream;
    n->stream = st;
    const vofp_status s = forward(n, r);
    n->stream = own;
    return s;
}
float* output(vofp_nn* n) { return n->out; }
// rms, its finish, input packing, ten convolutions, two poolings, two upsamplings, output layer
int forward_kernels(const vofp_nn*) { return 18; }
vofp_status read_device_error(vofp_nn* n) { return read_err(n); }
vofp_status train_from_grad_on(vofp_nn* n, cudaStream_t st, const float* dz, float lr, int update) {
    const cudaStream_t own = n->stream;
    n->stream = st;
    vofp_status s = backward(n, nullptr, dz);
    if (!s && update) adam(n, lr);
    n->stream = own;
    if (s) return s;
    return read_err(n);
}
vofp_status prepare_training(vofp_nn* n) { return ensure_grads(n); }
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
    if ((s = n->alloc(&n->derr, 1, n->allocs)) || cudaMemset(n->derr, 0, sizeof(int)) != cudaSuccess) {
        vofp_nn_destroy(n);
        return s ? s : VOFP_ERR_CUDA;
    }
    for (int i = 0; i < 10; ++i) {
        Layer l;
        l.cin = kLayers[i][0];
        l.cout = kLayers[i][1];
        l.cin_real = kLayers[i][2];
        l.nout_f = kLayers[i][3];
        l.nout_b = kLayers[i][4];
        auto& A = n->allocs;
        if ((s = n->alloc(&l.w, l.nw(), A)) || (s = n->alloc(&l.b, l.cout, A)) || (s = n->alloc(&l.gw, l.nw(), A)) ||
            (s = n->alloc(&l.gb, l.cout, A)) || (s = n->alloc(&l.mw, l.nw(), A)) || (s = n->alloc(&l.vw, l.nw(), A)) ||
            (s = n->alloc(&l.mb, l.cout, A)) || (s = n->alloc(&l.vb, l.cout, A)) ||
            (s = n->alloc(&l.blob_f, l.nw(), A)) || (s = n->alloc(&l.blob_b, l.nw(), A))) {
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
    auto& A = n->allocs;
    if ((s = n->alloc(&n->hw, 16, A)) || (s = n->alloc(&n->hb, 1, A)) || (s = n->alloc(&n->ghw, 16, A)) ||
        (s = n->alloc(&n->ghb, 1, A)) || (s = n->alloc(&n->mhw, 16, A)) || (s = n->alloc(&n->vhw, 16, A)) ||
        (s = n->alloc(&n->mhb, 1, A)) || (s = n->alloc(&n->vhb, 1, A)) || (s = n->alloc(&n->scal, 8, A))) {
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
    refresh_blobs(n);
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
    free_list(n->grad_allocs);
    free_list(n->grid_allocs);
    free_list(n->allocs);
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
    refresh_blobs(n);
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

vofp_status vofp_nn_conv_apply(vofp_nn* n, int layer, int data_grad, int nx, int ny, int nz, const uint16_t* in,
                               uint16_t* out) {
    if (!n || layer < 0 || layer >= 10 || nx <= 0 || ny <= 0 || nz <= 0 || !in || !out ||
        (reinterpret_cast<uintptr_t>(in) & 15) || (reinterpret_cast<uintptr_t>(out) & 15))
        return VOFP_ERR_INVALID_ARG;
    const Layer& l = n->L[layer];
    const bf16* x = reinterpret_cast<const bf16*>(in);
    bf16* y = reinterpret_cast<bf16*>(out);
    vofp_status s = data_grad ? conv(n, x, l.cout, l.blob_b, l.cin, l.nout_b, nullptr, false, y, 0, nx, ny, nz)
                              : conv(n, x, l.cin, l.blob_f, l.cout, l.nout_f, l.b, true, y, 0, nx, ny, nz);
    if (s) return s;
    return read_err(n);
}

vofp_status vofp_nn_conv_wgrad(vofp_nn* n, int layer, int nx, int ny, int nz, const uint16_t* x, const uint16_t* dy,
                               float* gw, float* gb) {
    if (!n || layer < 0 || layer >= 10 || nx <= 0 || ny <= 0 || nz <= 0 || !x || !dy || !gw || !gb ||
        (reinterpret_cast<uintptr_t>(x) & 15) || (reinterpret_cast<uintptr_t>(dy) & 15))
        return VOFP_ERR_INVALID_ARG;
    Layer l = n->L[layer];
    l.gw = gw;
    l.gb = gb;
    if (cudaMemsetAsync(gw, 0, sizeof(float) * l.nw(), n->stream) != cudaSuccess ||
        cudaMemsetAsync(gb, 0, sizeof(float) * l.cout, n->stream) != cudaSuccess)
        return VOFP_ERR_CUDA;
    vofp_status s = conv_wgrad(n, reinterpret_cast<const bf16*>(x), reinterpret_cast<const bf16*>(dy), l, nx, ny, nz);
    if (s) return s;
    return read_err(n);
}

vofp_status vofp_nn_train_step(vofp_nn* n, const float* r, const float* target, float lr, int update, float* loss) {
    if (!n || !r || !target) return VOFP_ERR_INVALID_ARG;
    if (!n->bound) {
        n->err = "no geometry bound";
        return VOFP_ERR_NOT_BUILT;
    }
    vofp_status s;
    if ((s = ensure_grads(n)) || (s = forward(n, r)) || (s = backward(n, target))) return s;
    if (update) adam(n, lr);
    if (loss) {
        if (cudaMemcpyAsync(loss, n->scal + 4, sizeof(float), cudaMemcpyDeviceToHost, n->stream) != cudaSuccess)
            return VOFP_ERR_CUDA;
    }
    if ((s = read_err(n))) return s;
    return cudaGetLastError() == cudaSuccess ? VOFP_OK : VOFP_ERR_CUDA;
}

}  // extern "C"
