// Host side of the TMA-fed red-black iteration: shared-memory opt-in, grid sizing, tensor maps and
// the launch.
#include <algorithm>

#include "vofp_rb_tma.cuh"

namespace vofp {
namespace {
constexpr int kRbStages = 3;
}

void prepare_rb_tma(vofp_ctx* c) {
    constexpr size_t smem = cg_rb_tma_smem<kRbStages>();
    cudaFuncSetAttribute(k_cg_rb_tma<kRbStages>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_cg_rb_tma<kRbStages>, kBX * kBY, smem) != cudaSuccess)
        nb = 0;
    cudaGetLastError();
    c->rb_tma_blocks_per_sm = nb;
    // same conditions as the FP32 TMA stencil (rows of 16-byte multiples, copies enabled)
    c->rb_tma_ok = c->tma_ok[0] && nb > 0;
}

bool launch_cg_rb_tma(vofp_ctx* c, cudaStream_t st, const float* r, const float* po, float* pn, float* xv, float* q) {
    using G = RbGeom;
    if (!c->rb_tma_ok || !c->Tzr) return false;
    const CUtensorMap *mr = tensor_map_f32(c, r, G::BW, kBY + 4), *mp = tensor_map_f32(c, po, G::BW, kBY + 4),
                      *mx = tensor_map_f32(c, c->Txf, G::BW, kBY + 2), *my = tensor_map_f32(c, c->Tyf, G::BW, kBY + 3),
                      *mz = tensor_map_f32(c, c->Tzr, G::BW, kBY + 2);
    if (!(mr && mp && mx && my && mz)) return false;
    RbMaps maps;
    maps.r = *mr;
    maps.p = *mp;
    maps.tx = *mx;
    maps.ty = *my;
    maps.tz = *mz;
    const long long tiles = (long long)ceil_div(c->d.nx, G::TW) * ceil_div(c->d.ny, kBY);
    int nb = 1, per = 1;
    // balanced split: the red-black step does more work per plane than the stencil, and with one
    // block per tile column too few warps per SM are left to cover it (measured 0.20 against
    // 0.17 ms at 512 x 256 x 128)
    plane_split(tiles, c->d.nz, (long long)num_sms() * c->rb_tma_blocks_per_sm, false, &nb, &per);
    launch_smem(c, k_cg_rb_tma<kRbStages>, dim3(nb), dim3(kBX, kBY), cg_rb_tma_smem<kRbStages>(), st, maps, c->d,
                per, po, pn, xv, q, c->sc, c->partials, c->counters);
    return true;
}

}  // namespace vofp
