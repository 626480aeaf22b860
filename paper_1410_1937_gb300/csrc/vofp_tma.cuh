// Tensor-memory-accelerator (TMA) plane pipeline for the CG stencil.
//
// The fused CG stencil (p = r + beta p_old, x += alpha p_old, t = (S A S) p, p.t) streams six
// arrays per cell and does little arithmetic, so its speed is set by how many bytes each SM keeps
// in flight.  Here every input plane of a block's 32 x 8 column tile is fetched by bulk tensor
// copies (cp.async.bulk.tensor, one elected thread) into a ring of NS shared-memory stages, each
// guarded by an mbarrier that counts the bytes landed; NS - 2 planes are in flight while the block
// computes.  Out-of-range boxes (x < 0, y < 0, z < 0 or past the end) are zero-filled by the copy
// engine, which is exactly the zero boundary value the stencil needs.
//
// Every wait on an mbarrier is bounded (about one second of wall time).  A wait that runs out
// sets VOFP_ERR_DEVICE_TIMEOUT in the iteration scalars, waits (bounded again) for the block's
// copies still in flight and leaves the loop; the solve then stops with that status.
#pragma once
#include <cuda.h>

#include "vofp_kernels.cuh"

namespace vofp {

// Work split of the plane-marching persistent kernels over `tiles` column tiles of nz planes and
// `resident` co-resident blocks.  column: one block per tile column (tiles <= resident), so all
// blocks march z in step and the halo rows a block reads from its neighbours' tiles were brought
// into L2 by those neighbours moments earlier.  Otherwise equal shares of tile-planes (in
// tile-major order) over all resident blocks.
inline void plane_split(long long tiles, int nz, long long resident, bool column, int* nb, int* per) {
    const long long total = tiles * nz;
    if (column && tiles <= resident) {
        *nb = (int)tiles;
        *per = nz;
        return;
    }
    *nb = (int)(resident < 1 ? 1 : (resident < total ? resident : total));
    *per = (int)((total + *nb - 1) / *nb);
}

// The six tensor maps of one CG stencil launch: r and p_old with a one-cell halo in x and y, Tx
// with a halo on the low-x side, Ty with a halo on the low-y side, Tz and x on the tile itself.
struct CgMaps {
    CUtensorMap r, p, tx, ty, tz, x;
};

// Box geometry per element type and cells per thread (CPT, along x): the tile is TW = 32 CPT by
// 8 cells.  The x start of every box is a multiple of 16 bytes (TMA rule): a halo box starts kHX
// cells left of the tile, so its width is TW + 2 kHX.  The p ring keeps CPT pad cells on each side
// of a row, so a thread's CPT own cells start at an index that is a multiple of CPT.
template <typename V, int CPT>
struct TmaGeom {
    static constexpr int TW = kBX * CPT;
    static constexpr int kHX = 16 / (int)sizeof(V);      // 4 (FP32) or 2 (FP64)
    static constexpr int kHW = TW + 2 * kHX;             // halo-box width
    static constexpr int kRN = kHW * (kBY + 2);          // r, p_old box (rows j0-1 .. j0+kBY)
    static constexpr int kXN = kHW * kBY;                // Tx box (rows j0 .. j0+kBY-1)
    static constexpr int kYN = TW * (kBY + 1);           // Ty box (rows j0-1 .. j0+kBY-1)
    static constexpr int kON = TW * kBY;                 // Tz, x boxes (the tile)
    static constexpr size_t al(size_t b) { return (b + 127) / 128 * 128; }
    static constexpr size_t oR = 0;
    static constexpr size_t oP = oR + al(kRN * sizeof(V));
    static constexpr size_t oX = oP + al(kRN * sizeof(V));
    static constexpr size_t oY = oX + al(kXN * sizeof(V));
    static constexpr size_t oZ = oY + al(kYN * sizeof(V));
    static constexpr size_t oV = oZ + al(kON * sizeof(V));
    static constexpr size_t kStage = oV + al(kON * sizeof(V));
    static constexpr uint32_t kTx = (uint32_t)((2 * kRN + kXN + kYN + 2 * kON) * sizeof(V));
    static constexpr int kPW = TW + 2 * CPT;             // p ring row: CPT pad cells each side
    static constexpr int kPN = kPW * (kBY + 2);
    static constexpr int kItems = kPN / CPT;             // form_p work items (CPT cells each)
};

template <typename V, int NS, int CPT>
constexpr size_t cg_tma_smem() {
    using G = TmaGeom<V, CPT>;
    return 128 + NS * G::kStage + 4 * G::kPN * sizeof(V) + NS * sizeof(uint64_t);
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// order this thread's earlier generic-proxy shared accesses before later async-proxy (TMA) ones
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
// Wait for the phase with the given parity to complete; false after about one second.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (unsigned it = 0;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 63u && global_ns() - t0 > 1000000000ull) return false;
    }
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

// Fused CG stencil (the ST_CG operation of k_stencil) with TMA-fed planes.  NS stages; the block
// marches its share of tile-planes like k_stencil.  Step k: wait for plane k+1; form
// p = r + beta p_old on it (one-cell halo) into a 4-plane ring; barrier; refill the stage of
// plane k-1 with plane k-1+NS; apply the stencil to plane k from the ring and stage k.  With
// CPT = 2 a thread owns two neighbouring cells in x and moves them as one 8-byte word.
template <typename V, int NS, int CPT>
__global__ void __launch_bounds__(kBX* kBY)
k_cg_tma(const __grid_constant__ CgMaps maps, const Dims d, const int per_block, V* __restrict__ pnew,
         V* __restrict__ xv, V* __restrict__ out, CgScalars* __restrict__ sc, double* __restrict__ partials,
         unsigned int* __restrict__ counter) {
    static_assert(CPT == 1 || (CPT == 2 && sizeof(V) == 4), "two cells per thread: FP32 only");
    using G = TmaGeom<V, CPT>;
    using Acc = typename AccFor<V>::type;
    using V2 = float2;
    constexpr int TW = G::TW, PW = G::kPW, HW = G::kHW, HX = G::kHX;
    extern __shared__ __align__(128) unsigned char tma_smem[];
    // bulk-copy destinations want 128-byte alignment: round the dynamic base up (128 bytes spare)
    unsigned char* smem_raw = tma_smem + ((128u - (smem_addr(tma_smem) & 127u)) & 127u);
    V* ring = reinterpret_cast<V*>(smem_raw + NS * G::kStage);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + NS * G::kStage + 4 * G::kPN * sizeof(V));
    __shared__ double sh[32];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + kBX * ty;
    const V beta = (V)sc->beta, alpha = (V)sc->alpha;
    Acc acc;
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t phase = 0u, pending = 0u;   // per stage: parity of the next wait; load in flight
    bool bad = false;
    auto stage = [&](int s) -> unsigned char* { return smem_raw + s * G::kStage; };
    auto rplane = [&](int kk) -> V* { return ring + ((kk + 4) & 3) * G::kPN; };
    // this thread's form_p items: ring index (multiple of CPT) and r/p box index of its first cell
    int f_dst[2], f_src[2];
    bool f_on[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int it = tid + q * kBX * kBY;
        f_on[q] = it < G::kItems;
        const int e = f_on[q] ? it * CPT : 0;
        const int ex = e % PW, ey = e / PW;
        f_dst[q] = e;
        f_src[q] = ey * HW + ex - CPT + HX;   // ring x index ex is the cell i0 + ex - CPT
    }
    const int xo = CPT * tx;                   // first own cell of this thread within the tile

    const int tiles_x = (d.nx + TW - 1) / TW;
    const long long ntiles = (long long)tiles_x * ((d.ny + kBY - 1) / kBY);
    const long long total = ntiles * d.nz;
    const long long w0 = min((long long)blockIdx.x * per_block, total);
    const long long w1 = min(w0 + per_block, total);
    for (long long w = w0; w < w1 && !bad;) {
        const long long tile_id = w / d.nz;
        const int k0 = int(w - tile_id * d.nz);
        const int k1 = (int)min((long long)d.nz, (long long)k0 + (w1 - w));
        w += k1 - k0;
        const int i0 = int(tile_id % tiles_x) * TW, j0 = int(tile_id / tiles_x) * kBY;
        const int i = i0 + xo, j = j0 + ty;
        // nx is even whenever CPT = 2 (rows of 16-byte multiples), so both cells share this flag
        const bool inside = i < d.nx && j < d.ny;
        auto slot = [&](int kk) { return (kk - k0 + 1) % NS; };
        // one thread issues the six box copies of plane kk into its stage
        auto issue = [&](int kk) {
            const int s = slot(kk);
            pending |= 1u << s;
            if (tid == 0) {
                unsigned char* b = stage(s);
                mbar_expect_tx(&bars[s], G::kTx);
                tma_load_3d(b + G::oR, &maps.r, &bars[s], i0 - HX, j0 - 1, kk);
                tma_load_3d(b + G::oP, &maps.p, &bars[s], i0 - HX, j0 - 1, kk);
                tma_load_3d(b + G::oX, &maps.tx, &bars[s], i0 - HX, j0, kk);
                tma_load_3d(b + G::oY, &maps.ty, &bars[s], i0, j0 - 1, kk);
                tma_load_3d(b + G::oZ, &maps.tz, &bars[s], i0, j0, kk);
                tma_load_3d(b + G::oV, &maps.x, &bars[s], i0, j0, kk);
            }
        };
        auto wait = [&](int kk) -> bool {
            const int s = slot(kk);
            const bool ok = mbar_wait_bounded(&bars[s], (phase >> s) & 1u);
            phase ^= 1u << s;
            pending &= ~(1u << s);
            return ok;
        };
        // p = r + beta p_old over plane kk's tile with its halo
        auto form_p = [&](int kk) {
            const unsigned char* b = stage(slot(kk));
            const V* R = reinterpret_cast<const V*>(b + G::oR);
            const V* P = reinterpret_cast<const V*>(b + G::oP);
            V* op = rplane(kk);
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                if (!f_on[q]) continue;
                if constexpr (CPT == 1) {
                    op[f_dst[q]] = fmav(beta, P[f_src[q]], R[f_src[q]]);
                } else {
                    const V2 pv = *reinterpret_cast<const V2*>(P + f_src[q]);
                    const V2 rv = *reinterpret_cast<const V2*>(R + f_src[q]);
                    *reinterpret_cast<V2*>(op + f_dst[q]) = make_float2(fmav(beta, pv.x, rv.x), fmav(beta, pv.y, rv.y));
                }
            }
        };

        // the previous segment's readers of the stages are done before they are refilled
        __syncthreads();
        if (tid == 0) fence_proxy_async_smem();
        const int last_pre = min(k0 - 2 + NS, k1);
        for (int kk = k0 - 1; kk <= last_pre; ++kk) issue(kk);
        const int oo = ty * TW + xo;          // own index in the Tz / x boxes
        bool ok = wait(k0 - 1);
        form_p(k0 - 1);
        V tzm1[CPT];
#pragma unroll
        for (int u = 0; u < CPT; ++u) tzm1[u] = reinterpret_cast<const V*>(stage(slot(k0 - 1)) + G::oZ)[oo + u];
        ok = wait(k0) && ok;
        form_p(k0);
        for (int k = k0; k < k1; ++k) {
            ok = wait(k + 1) && ok;
            form_p(k + 1);
            if (__syncthreads_or(!ok)) {
                bad = true;
                break;
            }
            if (k - 1 + NS <= k1) {
                if (tid == 0) fence_proxy_async_smem();
                issue(k - 1 + NS);
            }
            const unsigned char* b = stage(slot(k));
            const V* TX = reinterpret_cast<const V*>(b + G::oX);
            const V* TY = reinterpret_cast<const V*>(b + G::oY);
            const V* TZ = reinterpret_cast<const V*>(b + G::oZ);
            const V* PO = reinterpret_cast<const V*>(b + G::oP);
            const V* XO = reinterpret_cast<const V*>(b + G::oV);
            V tzk[CPT];
            const V* P0 = rplane(k);
            const V* Pp = rplane(k + 1);
            const V* Pm = rplane(k - 1);
            const int e = (ty + 1) * PW + xo + CPT;          // ring index of the first own cell
            const int ex = ty * HW + xo + HX;                 // Tx box index of the first own cell
            const int eb = (ty + 1) * HW + xo + HX;           // r / p_old box index of the first own cell
            const long long c = (long long)k * d.plane + i + (long long)d.nx * j;
            if constexpr (CPT == 1) {
                tzk[0] = TZ[oo];
                if (inside) {
                    const V v = P0[e];
                    V t = v;
                    t = fmav(-TX[ex], P0[e + 1], t);
                    t = fmav(-TX[ex - 1], P0[e - 1], t);
                    t = fmav(-TY[(ty + 1) * TW + xo], P0[e + PW], t);
                    t = fmav(-TY[ty * TW + xo], P0[e - PW], t);
                    t = fmav(-tzk[0], Pp[e], t);
                    t = fmav(-tzm1[0], Pm[e], t);
                    out[c] = t;
                    pnew[c] = v;
                    xv[c] = fmav(alpha, PO[eb], XO[oo]);
                    acc.add(v, t);
                }
            } else {
                const V2 tz2 = *reinterpret_cast<const V2*>(TZ + oo);
                tzk[0] = tz2.x;
                tzk[1] = tz2.y;
                if (inside) {
                    const V2 v = *reinterpret_cast<const V2*>(P0 + e);
                    const V lf = P0[e - 1], rt = P0[e + 2];
                    const V2 up = *reinterpret_cast<const V2*>(P0 + e + PW);
                    const V2 dn = *reinterpret_cast<const V2*>(P0 + e - PW);
                    const V2 zp = *reinterpret_cast<const V2*>(Pp + e);
                    const V2 zm = *reinterpret_cast<const V2*>(Pm + e);
                    const V2 txo = *reinterpret_cast<const V2*>(TX + ex);
                    const V txm = TX[ex - 1];
                    const V2 typ = *reinterpret_cast<const V2*>(TY + (ty + 1) * TW + xo);
                    const V2 tym = *reinterpret_cast<const V2*>(TY + ty * TW + xo);
                    V t0 = v.x, t1 = v.y;
                    t0 = fmav(-txo.x, v.y, t0);
                    t1 = fmav(-txo.y, rt, t1);
                    t0 = fmav(-txm, lf, t0);
                    t1 = fmav(-txo.x, v.x, t1);
                    t0 = fmav(-typ.x, up.x, t0);
                    t1 = fmav(-typ.y, up.y, t1);
                    t0 = fmav(-tym.x, dn.x, t0);
                    t1 = fmav(-tym.y, dn.y, t1);
                    t0 = fmav(-tzk[0], zp.x, t0);
                    t1 = fmav(-tzk[1], zp.y, t1);
                    t0 = fmav(-tzm1[0], zm.x, t0);
                    t1 = fmav(-tzm1[1], zm.y, t1);
                    const V2 po = *reinterpret_cast<const V2*>(PO + eb);
                    const V2 xold = *reinterpret_cast<const V2*>(XO + oo);
                    *reinterpret_cast<V2*>(out + c) = make_float2(t0, t1);
                    *reinterpret_cast<V2*>(pnew + c) = v;
                    *reinterpret_cast<V2*>(xv + c) = make_float2(fmav(alpha, po.x, xold.x), fmav(alpha, po.y, xold.y));
                    acc.add(v.x, t0);
                    acc.add(v.y, t1);
                }
            }
#pragma unroll
            for (int u = 0; u < CPT; ++u) tzm1[u] = tzk[u];
        }
    }
    if (bad) {
        // a copy did not land in time: record it, let the copies in flight finish, leave
        for (int s = 0; s < NS; ++s)
            if (pending & (1u << s)) mbar_wait_bounded(&bars[s], (phase >> s) & 1u);
        if (tid == 0) atomicCAS(&sc->status, (int)VOFP_OK, (int)VOFP_ERR_DEVICE_TIMEOUT);
    }
    double tot;
    if (grid_reduce(acc.value(), partials, counter, sh, &tot)) sc->pq_raw = tot;
}

}  // namespace vofp
