// Host side of the TMA-fed CG stencil: tensor maps (cuTensorMapEncodeTiled, looked up through the
// runtime), shared-memory opt-in, persistent grid sizing and the launch.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <cudaTypedefs.h>
#include <mutex>

#include "vofp_tma.cuh"

namespace vofp {

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime (null when the
// driver does not provide it)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

namespace {

// TMA stencil configurations: FP32 two cells per thread (64 x 8 tiles), FP64 one (32 x 8); both
// four stages, three resident blocks per SM.  VOFP_TMA_FP32_CPT=1 selects the 32 x 8 FP32 kernel
// with six stages (four blocks per SM).
constexpr int kTmaStages64 = 4;

// 3-D tensor map of one nx x ny x nz array with a box of bw x bh cells of one plane (cached).
// L2 promotion 64 B: the boxes' rows are 128-160 B, and wider promotion pulls neighbouring tiles'
// bytes from DRAM that are evicted before those tiles run (measured: 256 B promotion read 1.9x
// the algorithmic bytes and ran 25% slower on the FP32 stencil).
template <typename V>
const CUtensorMap* tensor_map(vofp_ctx* c, const V* ptr, int bw, int bh, int nxe = 0) {
    if (nxe <= 0) nxe = c->d.nx;
    const auto key = std::make_tuple((const void*)ptr, bw, bh * 65536 + (nxe == c->d.nx ? 0 : 1));
    auto it = c->tma_maps.find(key);
    if (it != c->tma_maps.end()) return &it->second;
    CUtensorMap m;
    std::memset(&m, 0, sizeof(m));
    const cuuint64_t dims[3] = {(cuuint64_t)nxe, (cuuint64_t)c->d.ny, (cuuint64_t)c->d.nz};
    const cuuint64_t strides[2] = {(cuuint64_t)nxe * sizeof(V), (cuuint64_t)nxe * c->d.ny * sizeof(V)};
    const cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)bh, 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    const CUresult r = tensor_map_encoder()(
        &m, sizeof(V) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
        const_cast<V*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
        CU_TENSOR_MAP_L2_PROMOTION_L2_64B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return nullptr;
    return &(c->tma_maps[key] = m);
}

template <typename V, int NS, int CPT>
bool launch_tma(vofp_ctx* c, cudaStream_t st, const V* Tx, const V* Ty, const V* Tz, const V* r, const V* po,
                   V* pn, V* xv, V* q, bool column = false) {
    using G = TmaGeom<V, CPT>;
    const CUtensorMap *mr = tensor_map(c, r, G::kHW, kBY + 2), *mp = tensor_map(c, po, G::kHW, kBY + 2),
                      *mx = tensor_map(c, Tx, G::kHW, kBY), *my = tensor_map(c, Ty, G::TW, kBY + 1),
                      *mz = tensor_map(c, Tz, G::TW, kBY), *mv = tensor_map(c, (const V*)xv, G::TW, kBY);
    if (!(mr && mp && mx && my && mz && mv)) return false;
    CgMaps maps;
    maps.r = *mr;
    maps.p = *mp;
    maps.tx = *mx;
    maps.ty = *my;
    maps.tz = *mz;
    maps.x = *mv;
    const long long tiles = (long long)ceil_div(c->d.nx, G::TW) * ceil_div(c->d.ny, kBY);
    const int f64 = sizeof(V) == 8 ? 1 : 0;
    int nb = 1, per = 1;
    const int per_sm = (sizeof(V) == 4 && NS == 6 && CPT == 2) ? c->tma_blocks_deep32 : c->tma_blocks_per_sm[f64];
    plane_split(tiles, c->d.nz, (long long)num_sms() * per_sm, column, &nb, &per);
    launch_smem(c, k_cg_tma<V, NS, CPT>, dim3(nb), dim3(kBX, kBY), cg_tma_smem<V, NS, CPT>(), st, maps, c->d, per,
                pn, xv, q, c->sc, c->partials, c->counters);
    return true;
}

}  // namespace

const CUtensorMap* tensor_map_f32(vofp_ctx* c, const float* ptr, int bw, int bh) {
    return tensor_map_encoder() ? tensor_map(c, ptr, bw, bh) : nullptr;
}
const CUtensorMap* tensor_map_f32_x(vofp_ctx* c, const float* ptr, int nxe, int bw, int bh) {
    if (!tensor_map_encoder() || (nxe * sizeof(float)) % 16 != 0) return nullptr;
    return tensor_map(c, ptr, bw, bh, nxe);
}

template <typename V>
bool launch_cg_tma(vofp_ctx* c, cudaStream_t st, const V* Tx, const V* Ty, const V* Tz, const V* r, const V* po,
                   V* pn, V* xv, V* q) {
    if constexpr (sizeof(V) == 8) {
        return c->tma_ok[1] && launch_tma<double, kTmaStages64, 1>(c, st, Tx, Ty, Tz, r, po, pn, xv, q);
    } else {
        if (!c->tma_ok[0]) return false;
        if (c->tma_cpt32 == 1) return launch_tma<float, 6, 1>(c, st, Tx, Ty, Tz, r, po, pn, xv, q);
        // Column split with six stages when the tile columns fill, without exceeding, one wave of
        // the six-stage kernel (two blocks per SM): every block marches a whole column in step with
        // its neighbours (halo rows from L2, four planes in flight per block; measured 0.096 against
        // 0.117 ms for the balanced four-stage split at 512 x 256 x 128).  Otherwise the balanced
        // four-stage split (small grids live in L2; large grids need several columns per block).
        const long long tiles = (long long)ceil_div(c->d.nx, 2 * kBX) * ceil_div(c->d.ny, kBY);
        const long long deep = (long long)num_sms() * c->tma_blocks_deep32;
        if (deep > 0 && tiles <= deep && 2 * tiles > deep)
            return launch_tma<float, 6, 2>(c, st, Tx, Ty, Tz, r, po, pn, xv, q, true);
        return launch_tma<float, 4, 2>(c, st, Tx, Ty, Tz, r, po, pn, xv, q, false);
    }
}
template bool launch_cg_tma<float>(vofp_ctx*, cudaStream_t, const float*, const float*, const float*, const float*,
                                   const float*, float*, float*, float*);
template bool launch_cg_tma<double>(vofp_ctx*, cudaStream_t, const double*, const double*, const double*,
                                    const double*, const double*, double*, double*, double*);

// Opt the TMA stencil kernels into their dynamic shared memory, size their persistent grids and
// decide per precision whether the tensor maps can be built.
void prepare_tma(vofp_ctx* c) {
    const char* env = std::getenv("VOFP_STENCIL_TMA");
    const bool tma_allowed = !(env && std::strcmp(env, "0") == 0) && tensor_map_encoder() != nullptr;
    const char* cpt = std::getenv("VOFP_TMA_FP32_CPT");
    c->tma_cpt32 = (cpt && std::strcmp(cpt, "1") == 0) ? 1 : 2;
    constexpr size_t sb = cg_tma_smem<float, 6, 1>(), sd = cg_tma_smem<double, kTmaStages64, 1>();
    constexpr size_t s4 = cg_tma_smem<float, 4, 2>(), s6 = cg_tma_smem<float, 6, 2>();
    cudaFuncSetAttribute(k_cg_tma<float, 4, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s4);
    cudaFuncSetAttribute(k_cg_tma<float, 6, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s6);
    cudaFuncSetAttribute(k_cg_tma<float, 6, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb);
    cudaFuncSetAttribute(k_cg_tma<double, kTmaStages64, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sd);
    int b32 = 0, b64 = 0, bdeep = 0;
    cudaError_t e32 = c->tma_cpt32 == 1
                          ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b32, k_cg_tma<float, 6, 1>, kBX * kBY, sb)
                          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b32, k_cg_tma<float, 4, 2>, kBX * kBY, s4);
    if (e32 != cudaSuccess) b32 = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bdeep, k_cg_tma<float, 6, 2>, kBX * kBY, s6) != cudaSuccess)
        bdeep = 0;
    c->tma_blocks_deep32 = bdeep;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b64, k_cg_tma<double, kTmaStages64, 1>, kBX * kBY, sd) !=
        cudaSuccess)
        b64 = 0;
    cudaGetLastError();
    c->tma_blocks_per_sm[0] = b32;
    c->tma_blocks_per_sm[1] = b64;
    // the tensor maps need row and plane pitches that are multiples of 16 bytes
    c->tma_ok[0] = tma_allowed && b32 > 0 && (c->d.nx * sizeof(float)) % 16 == 0;
    c->tma_ok[1] = tma_allowed && b64 > 0 && (c->d.nx * sizeof(double)) % 16 == 0;
}

}  // namespace vofp
