// Host side of the TMA-fed red-black iteration: shared-memory opt-in, grid sizing, tensor maps and
// the launch.
#include <algorithm>

#include "vofp_rb_tma.cuh"

namespace vofp {
namespace {
constexpr int kRbStages = 3;

template <int TH>
int prepare_th() {
    constexpr size_t smem = cg_rb_tma_smem<kRbStages, TH>();
    cudaFuncSetAttribute(k_cg_rb_tma<kRbStages, TH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_cg_rb_tma<kRbStages, TH>, kBX * TH, smem) != cudaSuccess)
        nb = 0;
    cudaGetLastError();
    return nb;
}

template <int TH>
bool launch_th(vofp_ctx* c, cudaStream_t st, const float* r, const float* po, float* pn, float* xv, float* q,
               int per_sm, bool column) {
    using G = RbGeom<TH>;
    const CUtensorMap *mr = tensor_map_f32(c, r, G::BW, TH + 4), *mp = tensor_map_f32(c, po, G::BW, TH + 4),
                      *mx = tensor_map_f32(c, c->Txf, G::BW, TH + 2), *my = tensor_map_f32(c, c->Tyf, G::BW, TH + 3),
                      *mz = tensor_map_f32(c, c->Tzr, G::BW, TH + 2);
    if (!(mr && mp && mx && my && mz)) return false;
    RbMaps maps;
    maps.r = *mr;
    maps.p = *mp;
    maps.tx = *mx;
    maps.ty = *my;
    maps.tz = *mz;
    const long long tiles = (long long)ceil_div(c->d.nx, G::TW) * ceil_div(c->d.ny, TH);
    int nb = 1, per = 1;
    plane_split(tiles, c->d.nz, (long long)num_sms() * per_sm, column, &nb, &per);
    launch_smem(c, k_cg_rb_tma<kRbStages, TH>, dim3(nb), dim3(kBX, TH), cg_rb_tma_smem<kRbStages, TH>(), st, maps,
                c->d, per, po, pn, xv, q, c->sc, c->partials, c->counters);
    return true;
}
}  // namespace

void prepare_rb_tma(vofp_ctx* c) {
    const int nb = prepare_th<8>();
    c->rb_tma_blocks_per_sm = nb;
    // same conditions as the FP32 TMA stencil (rows of 16-byte multiples, copies enabled)
    c->rb_tma_ok = c->tma_ok[0] && nb > 0;
}

bool launch_cg_rb_tma(vofp_ctx* c, cudaStream_t st, const float* r, const float* po, float* pn, float* xv, float* q) {
    if (!c->rb_tma_ok || !c->Tzr) return false;
    // 64 x 8 tiles, balanced split of tile-planes over three resident blocks per SM: the red-black
    // step does more work per plane than the stencil, and neither one block per tile column
    // (0.204 ms at 512 x 256 x 128) nor 64 x 4 tiles (0.216 ms balanced, 0.228 ms by column) beat
    // it (0.170 ms)
    return launch_th<8>(c, st, r, po, pn, xv, q, c->rb_tma_blocks_per_sm, false);
}

}  // namespace vofp
