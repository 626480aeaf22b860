// Host side and small kernels of the colour-compact red-black inner solve (see vofp_rbc.cuh).
//
// Per operator (on the device, deterministic order):
//   exceptions  even-parity cells with an unknown that are not red (members of merge groups),
//               sorted by cell index; their compact index is N/2 + e;
//   exception tables  per exception the black pair behind each face and the face coefficient;
//   fix rows    black cells next to an exception, sorted, with the exception index and the face
//               coefficient behind each of their six faces (-1 / 0 where there is none);
//   bits        compact entries that hold a copy of a group value (excluded from the dots);
//   gref, gfx   the compact index and the fix-row index (-1 if none) of every entry of the
//               merge-group cell lists.
// Per iteration: the TMA iteration kernel (every even cell takes the red formula), the fix kernel
// (exception entries; black rows next to an exception get the exception's p in place of the red
// formula; merge groups summed and their value written to every member) and the vector update on
// the compact vectors.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "vofp_rbc.cuh"

namespace vofp {
namespace {

constexpr int kNT = 256;
constexpr int kRbcStages = 3;
// the iteration kernel's and the fix rows' block partials of p.Ap live in the last quarter of the
// partials buffer (no other reduction of an inner iteration uses it)
constexpr int kPqBase = 3 * (kMaxPartials / 4);
constexpr int kChunk = 2048;            // cells per block of the compaction passes (8 per thread)

int grid_n(long long n) {
    long long b = (n + kNT - 1) / kNT;
    return int(std::max(1LL, std::min(b, (long long)num_sms() * 8)));
}

__device__ __forceinline__ bool bit_of(const uint32_t* __restrict__ bits, long long c) {
    return (bits[c >> 5] >> (c & 31)) & 1u;
}
__device__ __forceinline__ int parity(const Dims& d, long long c) {
    int i, j, k;
    cell_ijk(d, c, i, j, k);
    return (i + j + k) & 1;
}
// black (odd-parity) cell of pair h (nx even: the pair's cells are 2h and 2h+1)
__device__ __forceinline__ long long black_of(const Dims& d, long long h) {
    const long long row = h / (d.nx >> 1);
    const int j = int(row % d.ny), k = int(row / d.ny);
    return 2 * h + 1 - ((j + k) & 1);
}
// exception: even parity, an unknown, not red
__device__ __forceinline__ bool is_exception(const Dims& d, long long c, const int32_t* root, const uint32_t* red) {
    return root[c] >= 0 && parity(d, c) == 0 && !bit_of(red, c);
}
// fix row: black cell with an exception behind one of its faces
__device__ __forceinline__ bool is_fix_row(const Dims& d, long long c, const uint8_t* isexc) {
    if (parity(d, c) == 0) return false;
    int i, j, k;
    cell_ijk(d, c, i, j, k);
    return (i > 0 && isexc[c - 1]) || (i < d.nx - 1 && isexc[c + 1]) || (j > 0 && isexc[c - d.nx]) ||
           (j < d.ny - 1 && isexc[c + d.nx]) || (k > 0 && isexc[c - d.plane]) || (k < d.nz - 1 && isexc[c + d.plane]);
}

template <int MODE>
__device__ __forceinline__ bool pred(const Dims& d, long long c, const int32_t* root, const uint32_t* red,
                                     const uint8_t* isexc) {
    if (MODE == 0) return is_exception(d, c, root, red);
    return is_fix_row(d, c, isexc);
}

// stable compaction, pass 1: count per chunk of kChunk cells
template <int MODE>
__global__ void __launch_bounds__(kNT) k_cmp_count(Dims d, const int32_t* __restrict__ root,
                                                   const uint32_t* __restrict__ red, const uint8_t* __restrict__ isexc,
                                                   unsigned int* __restrict__ counts) {
    __shared__ unsigned int sh[kNT / 32];
    const long long c0 = (long long)blockIdx.x * kChunk + (long long)threadIdx.x * (kChunk / kNT);
    unsigned int n = 0;
    for (int u = 0; u < kChunk / kNT; ++u) {
        const long long c = c0 + u;
        if (c < d.n && pred<MODE>(d, c, root, red, isexc)) ++n;
    }
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = n;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int s = 0;
        for (int w = 0; w < kNT / 32; ++w) s += sh[w];
        counts[blockIdx.x] = s;
    }
}

// pass 2: exclusive scan of the chunk counts (one block), total into counts[nchunks]
__global__ void k_cmp_scan(int nchunks, unsigned int* __restrict__ counts, unsigned int* __restrict__ offsets) {
    __shared__ unsigned int part[1024];
    const int t = threadIdx.x, per = (nchunks + 1023) / 1024;
    unsigned int s = 0;
    for (int u = 0; u < per; ++u) {
        const int i = t * per + u;
        if (i < nchunks) s += counts[i];
    }
    part[t] = s;
    __syncthreads();
    if (t == 0) {
        unsigned int run = 0;
        for (int i = 0; i < 1024; ++i) {
            const unsigned int v = part[i];
            part[i] = run;
            run += v;
        }
        counts[nchunks] = run;
    }
    __syncthreads();
    unsigned int run = part[t];
    for (int u = 0; u < per; ++u) {
        const int i = t * per + u;
        if (i < nchunks) {
            offsets[i] = run;
            run += counts[i];
        }
    }
}

// pass 3: write the selected cells of each chunk in index order
template <int MODE>
__global__ void __launch_bounds__(kNT) k_cmp_write(Dims d, const int32_t* __restrict__ root,
                                                   const uint32_t* __restrict__ red, const uint8_t* __restrict__ isexc,
                                                   const unsigned int* __restrict__ offsets, int* __restrict__ out) {
    __shared__ unsigned int sh[kNT / 32];
    const long long c0 = (long long)blockIdx.x * kChunk + (long long)threadIdx.x * (kChunk / kNT);
    unsigned int n = 0;
    for (int u = 0; u < kChunk / kNT; ++u) {
        const long long c = c0 + u;
        if (c < d.n && pred<MODE>(d, c, root, red, isexc)) ++n;
    }
    // exclusive scan of n over the block's threads (in thread order = cell order)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned int x = n;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    unsigned int wbase = 0;
    for (int w = 0; w < wid; ++w) wbase += sh[w];
    unsigned int pos = offsets[blockIdx.x] + wbase + x - n;
    for (int u = 0; u < kChunk / kNT; ++u) {
        const long long c = c0 + u;
        if (c < d.n && pred<MODE>(d, c, root, red, isexc)) out[pos++] = (int)c;
    }
}

__global__ void k_mark(int n, const int* __restrict__ cells, uint8_t* __restrict__ flag, uint8_t v) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) flag[cells[t]] = v;
}

// index of cell c in a sorted cell list (or -1)
__device__ __forceinline__ int find_sorted(const int* __restrict__ list, int n, long long c) {
    int lo = 0, hi = n - 1;
    while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        const long long v = list[mid];
        if (v == c) return mid;
        if (v < c) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}
__device__ __forceinline__ int find_exc(const int* __restrict__ exc, int ne, long long c) {
    return find_sorted(exc, ne, c);
}

// coefficient of face f (order +x, -x, +y, -y, +z, -z) of cell c: the + face of the lower cell
__device__ __forceinline__ float face_T(const Dims& d, long long c, int f, const float* __restrict__ Tx,
                                        const float* __restrict__ Ty, const float* __restrict__ Tz) {
    switch (f) {
        case 0: return Tx[c];
        case 1: return Tx[c - 1];
        case 2: return Ty[c];
        case 3: return Ty[c - d.nx];
        case 4: return Tz[c];
        default: return Tz[c - d.plane];
    }
}

// per exception: the compact index of the black pair behind each face and the face coefficient
// (the own pair and 0 at the domain boundary), in the order of the red formula
__global__ void k_exc_tables(Dims d, int ne, const int* __restrict__ exc, const float* __restrict__ Tx,
                             const float* __restrict__ Ty, const float* __restrict__ Tz, int* __restrict__ enb,
                             float* __restrict__ eT) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    const long long ce = exc[e];
    int i, j, k;
    cell_ijk(d, ce, i, j, k);
    const bool has[6] = {i < d.nx - 1, i > 0, j < d.ny - 1, j > 0, k < d.nz - 1, k > 0};
    const long long nb[6] = {ce + 1, ce - 1, ce + d.nx, ce - d.nx, ce + d.plane, ce - d.plane};
    for (int f = 0; f < 6; ++f) {
        enb[6 * e + f] = (int)((has[f] ? nb[f] : ce) >> 1);
        eT[6 * e + f] = has[f] ? face_T(d, ce, f, Tx, Ty, Tz) : 0.0f;
    }
}

// per fix row: the exception index and the face coefficient behind each face (ne, whose
// difference entry is 0, and 0 where there is none), and its compact index (-1 for a merge-group
// member: its group handles it).  Row nf is a dummy with no exception.
__global__ void k_fix_faces(Dims d, int nf, const int* __restrict__ fcell, const int* __restrict__ exc, int ne,
                            const uint8_t* __restrict__ isexc, const uint8_t* __restrict__ isgrp,
                            const float* __restrict__ Tx, const float* __restrict__ Ty, const float* __restrict__ Tz,
                            int* __restrict__ fexc, float* __restrict__ fT, int* __restrict__ fh) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r > nf) return;
    if (r == nf) {
        for (int f = 0; f < 6; ++f) {
            fexc[6 * r + f] = ne;
            fT[6 * r + f] = 0.0f;
        }
        return;
    }
    const long long b = fcell[r];
    int i, j, k;
    cell_ijk(d, b, i, j, k);
    const long long nb[6] = {i < d.nx - 1 ? b + 1 : -1, i > 0 ? b - 1 : -1,
                             j < d.ny - 1 ? b + d.nx : -1, j > 0 ? b - d.nx : -1,
                             k < d.nz - 1 ? b + d.plane : -1, k > 0 ? b - d.plane : -1};
    for (int f = 0; f < 6; ++f) {
        const int e = (nb[f] >= 0 && isexc[nb[f]]) ? find_exc(exc, ne, nb[f]) : -1;
        fexc[6 * r + f] = e >= 0 ? e : ne;
        fT[6 * r + f] = e >= 0 ? face_T(d, b, f, Tx, Ty, Tz) : 0.0f;
    }
    fh[r] = isgrp[b] ? -1 : (int)(b >> 1);
}

// compact index and fix-row index (-1 if none) of every merge-group cell entry
__global__ void k_gref(Dims d, int n, const int* __restrict__ gcells, const int* __restrict__ exc, int ne,
                       const int* __restrict__ fcell, int nf, long long nh, int* __restrict__ gref,
                       int* __restrict__ gfx) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const long long c = gcells[t];
    const bool black = parity(d, c) != 0;
    gref[t] = black ? (int)(c >> 1) : (int)(nh + find_exc(exc, ne, c));
    gfx[t] = black ? find_sorted(fcell, nf, c) : -1;
}

// per merge group: the compact and fix-row indices of up to four members (padding: the master
// and the dummy fix row nf; a member that is no fix row also gets nf) and the member count
__global__ void k_gflat(int ng, const int* __restrict__ gptr, const int* __restrict__ gref,
                        const int* __restrict__ gfx, int nf, int4* __restrict__ gm, int4* __restrict__ gf,
                        int* __restrict__ gn) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ng) return;
    const int u0 = gptr[g], n = gptr[g + 1] - u0;
    int m[4], f[4];
    for (int u = 0; u < 4; ++u) {
        m[u] = gref[u0 + (u < n ? u : 0)];
        f[u] = (u < n && gfx[u0 + u] >= 0) ? gfx[u0 + u] : nf;
    }
    gm[g] = make_int4(m[0], m[1], m[2], m[3]);
    gf[g] = make_int4(f[0], f[1], f[2], f[3]);
    gn[g] = n;
}

// compact dot-exclusion bits: the entry's cell belongs to another cell's group (or has no unknown)
__global__ void k_cbits(Dims d, long long nh, int ne, const int* __restrict__ exc, const int32_t* __restrict__ root,
                        uint32_t* __restrict__ bits) {
    const long long nc = nh + ne, nw = (nc + 31) / 32;
    for (long long wd = blockIdx.x * (long long)blockDim.x + threadIdx.x; wd < nw; wd += (long long)gridDim.x * blockDim.x) {
        uint32_t v = 0;
        for (int u = 0; u < 32; ++u) {
            const long long t = wd * 32 + u;
            if (t >= nc) break;
            const long long c = t < nh ? black_of(d, t) : (long long)exc[t - nh];
            if (root[c] != (int32_t)c) v |= 1u << u;
        }
        bits[wd] = v;
    }
}

// inner start: gather the FP64 reduced right-hand side (full grid) onto the compact vectors,
// normalised; x = 0; p_old = 0 unless the direction is kept; r.r over the entries that count
__global__ void k_rbc_prep(Dims d, long long nh, int ne, const int* __restrict__ exc, const double* __restrict__ src,
                           const uint32_t* __restrict__ bits, float* __restrict__ r, float* __restrict__ x,
                           float* __restrict__ p0, CgScalars* sc, double* __restrict__ partials,
                           unsigned int* __restrict__ counter) {
    __shared__ double sh[32];
    const double rr = sc->rr0;
    const double inv = (rr > 0.0 && !sc->done) ? 1.0 / sqrt(rr) : 0.0;
    const bool keep = sc->keep_dir && sc->dir_valid;
    AccF2 acc;
    const long long nc = nh + ne;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nc; t += (long long)gridDim.x * blockDim.x) {
        const long long c = t < nh ? black_of(d, t) : (long long)exc[t - nh];
        const float v = (float)(src[c] * inv);
        r[t] = v;
        x[t] = 0.0f;
        if (!keep) p0[t] = 0.0f;
        if (!bit_of(bits, t)) acc.add(v, v);
    }
    double tot;
    if (grid_reduce(acc.value(), partials, counter, sh, &tot)) inner_start_scalars(sc, tot, rr, keep);
}

// correction of fix row rr: the black row took the red formula at each neighbouring exception,
// T_f (w_red - p_e) puts the exception's p back (faces without one point at a zero entry)
__device__ __forceinline__ float fix_delta(int rr, const int* __restrict__ fexc, const float* __restrict__ fT,
                                           const float* __restrict__ dE) {
    int e[6];
    float T[6];
#pragma unroll
    for (int f = 0; f < 6; ++f) {
        e[f] = fexc[6 * rr + f];
        T[f] = fT[6 * rr + f];
    }
    float delta = 0.0f;
#pragma unroll
    for (int f = 0; f < 6; ++f) delta = fmav(T[f], dE[e[f]], delta);
    return delta;
}

// After the iteration kernel (which also forms the exception rows and dE).  Fix rows that are not
// merge-group members (threads 0..nf-1): q += delta.
// Merge groups (threads nf..nf+ng-1): every member's final row (the exception row, or the black
// row plus its correction), then the group value sum + gcorr p_G written to every member.
// p.delta of the corrections and gcorr p_G^2 as this block's partial of p.Ap (after the iteration
// kernel's partials), which the update kernel sums.
__global__ void __launch_bounds__(kNT)
k_rbc_fix_rows(int nf, int ng, const int* __restrict__ fh, const int* __restrict__ fexc,
               const float* __restrict__ fT, const float* __restrict__ dE, const int4* __restrict__ gm,
               const int4* __restrict__ gf, const int* __restrict__ gn, const int* __restrict__ gptr,
               const int* __restrict__ gref, const int* __restrict__ gfx, const double* __restrict__ gcorr,
               const float* __restrict__ pn, float* __restrict__ q, double* __restrict__ pq_part) {
    __shared__ double sh[32];
    grid_dep_wait();
    grid_dep_trigger();
    AccF2 acc;
    double corr = 0.0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nf + ng; t += gridDim.x * blockDim.x) {
        if (t < nf) {
            const int h = fh[t];
            if (h >= 0) {
                const float delta = fix_delta(t, fexc, fT, dE);
                q[h] += delta;
                acc.add(pn[h], delta);
            }
            continue;
        }
        const int g = t - nf, n = gn[g];
        const int4 m4 = gm[g], f4 = gf[g];
        const double gc = gcorr[g];
        const double pm = (double)pn[m4.x];
        double s = 0.0;
        if (n <= 4) {
            const int mm[4] = {m4.x, m4.y, m4.z, m4.w}, ff[4] = {f4.x, f4.y, f4.z, f4.w};
            float qv[4], pv[4], dv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                qv[u] = q[mm[u]];
                pv[u] = pn[mm[u]];
                dv[u] = fix_delta(ff[u], fexc, fT, dE);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (u < n) {
                    s += (double)(qv[u] + dv[u]);
                    acc.add(pv[u], dv[u]);
                }
            const float qm = (float)(s + gc * pm);
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (u < n) q[mm[u]] = qm;
        } else {
            const int u0 = gptr[g], u1 = gptr[g + 1];
            for (int u = u0; u < u1; ++u) {
                const int ix = gref[u], fr = gfx[u] >= 0 ? gfx[u] : nf;
                const float dv = fix_delta(fr, fexc, fT, dE);
                s += (double)(q[ix] + dv);
                acc.add(pn[ix], dv);
            }
            const float qm = (float)(s + gc * pm);
            for (int u = u0; u < u1; ++u) q[gref[u]] = qm;
        }
        corr += gc * pm * pm;
    }
    // this block's p.delta and group terms (fixed order); the update kernel sums the partials
    const double v = warp_sum(acc.value() + corr);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += sh[w];
        pq_part[blockIdx.x] = b;
    }
}

// end of an inner solve: x_f (full grid) = x + alpha p_old of the compact vectors (black cells),
// 0 on even cells; then the exceptions
__global__ void k_rbc_expand(Dims d, const float* __restrict__ x, const float* __restrict__ p0,
                             float* __restrict__ xf, const CgScalars* sc) {
    const float alpha = (float)sc->alpha;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < d.n; c += (long long)gridDim.x * blockDim.x)
        xf[c] = parity(d, c) ? __fmaf_rn(alpha, p0[c >> 1], x[c >> 1]) : 0.0f;
}
__global__ void k_rbc_expand_exc(long long nh, int ne, const int* __restrict__ exc, const float* __restrict__ x,
                                 const float* __restrict__ p0, float* __restrict__ xf, const CgScalars* sc) {
    const float alpha = (float)sc->alpha;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < ne) xf[exc[e]] = __fmaf_rn(alpha, p0[nh + e], x[nh + e]);
}

// Split of the iteration kernel's work over at most `slots` resident blocks. The tiles form groups
// of gx x gy neighbours (gx dividing the tile columns along x, gy the tile rows); the blocks of a
// group march the same planes in the same steps, one tile each. Group g takes the items
// [g per, (g+1) per) of w = column * (nz + pad) + pad + plane over the group columns (x-fastest),
// so that every column starts with `pad` items that stand for no plane. Three things set the
// kernel's time:
//  - its costliest block: a block marches each column segment it holds with kSegSteps plane steps
//    besides its planes (four prologue steps that fill the p and w rings before the first output
//    plane, and the two closing t steps); padding charges a column's first segment for them in the
//    split itself, so that fewer blocks pay for two segments;
//  - whether the tiles on either side of a group edge are marched at the same plane in the same
//    step, so that the halo of their boxes comes from L2. Inside a group that always holds; across
//    an x edge (the next column, nz + pad items on) or a y edge (ncx columns on) it holds when that
//    distance is within kAlignSteps of a multiple of per. Otherwise the halo of that edge comes
//    from DRAM. Measured at 512x256x128 with 32 x 16 tiles (DRAM bytes of one launch for three
//    groupings, fitted per misaligned edge): 9.7 B per cell when every x edge is apart (the x halo
//    is two partial sectors per box row on each side), 3.5 B per cell when every y edge is (two
//    rows of r and p_old, seven coefficient rows), against 24 B per cell of the iteration itself;
//  - the slots a group size leaves unused (slots / (gx gy) groups).
// Candidates: every (gx, gy) with gx gy <= kMaxGroup, pad 0 .. 2 kSegSteps, per from the fewest
// items that fit in the groups up to four more; score = costliest block x (1 + the DRAM bytes of
// the misaligned edges' halo per 24 B); ties keep the smaller group, pad, per.
// VOFP_RBC_GROUP="gx,gy" fixes the group (when both divide).
constexpr int kSegSteps = 6;
constexpr long long kAlignSteps = 3;
constexpr double kHaloX = 9.7 / 24.0, kHaloY = 3.5 / 24.0;
constexpr long long kMaxGroup = 16;

long long split_cost(long long cols, long long nz, long long per, int pad, long long* nb) {
    const long long nzp = nz + pad, total = cols * nzp;
    long long worst = 0, groups = 0;
    for (long long w0 = 0; w0 < total; w0 += per, ++groups) {
        const long long w1 = std::min(w0 + per, total);
        long long cost = 0;
        for (long long w = w0; w < w1;) {
            const long long t = w / nzp, kp0 = w - t * nzp, kp1 = std::min(nzp, kp0 + (w1 - w));
            w += kp1 - kp0;
            const long long k0 = std::max(kp0 - pad, 0LL), k1 = kp1 - pad;
            if (k1 > k0) cost += (k1 - k0) + kSegSteps;
        }
        worst = std::max(worst, cost);
    }
    *nb = groups;
    return worst;
}

bool aligned(long long dist_items, long long per) {
    const long long r = dist_items % per;
    return std::min(r, per - r) <= kAlignSteps;
}

void rbc_split(long long tiles_x, long long tiles_y, long long nz, long long slots, int force_gx, int force_gy,
               RbcSplit* out, int* nblocks) {
    double best = 0.0;
    bool have = false;
    for (long long gy = 1; gy <= tiles_y && gy <= kMaxGroup; ++gy) {
        if (tiles_y % gy) continue;
        for (long long gx = 1; gx <= tiles_x && gx * gy <= kMaxGroup; ++gx) {
            if (tiles_x % gx || gx * gy > slots) continue;
            if (force_gx > 0 && (gx != force_gx || gy != force_gy)) continue;
            const long long ncx = tiles_x / gx, ncy = tiles_y / gy, cols = ncx * ncy, gslots = slots / (gx * gy);
            for (int pad = 0; pad <= 2 * kSegSteps; ++pad) {
                const long long nzp = nz + pad, total = cols * nzp;
                const long long pmin = std::max(1LL, (total + gslots - 1) / gslots);
                for (long long per = pmin; per <= pmin + 4 && per <= total; ++per) {
                    // fraction of the x and y tile edges whose two sides drift apart
                    const double fx = (ncx > 1 && !aligned(nzp, per)) ? double(ncx - 1) / double(tiles_x - 1) : 0.0;
                    const double fy =
                        (ncy > 1 && !aligned(ncx * nzp, per)) ? double(ncy - 1) / double(tiles_y - 1) : 0.0;
                    long long ng = 0;
                    const double score = (double)split_cost(cols, nz, per, pad, &ng) * (1.0 + kHaloX * fx + kHaloY * fy);
                    if (!have || score < best) {
                        have = true;
                        best = score;
                        *nblocks = (int)(ng * gx * gy);
                        *out = RbcSplit{(int)per, pad, (int)gx, (int)gy};
                    }
                }
            }
        }
    }
}

bool parse_group(int* gx, int* gy) {
    const char* env = std::getenv("VOFP_RBC_GROUP");
    *gx = *gy = 0;
    if (!env) return false;
    int a = 0, b = 0;
    if (std::sscanf(env, "%d,%d", &a, &b) != 2 || a < 1 || b < 1) return false;
    *gx = a;
    *gy = b;
    return true;
}

}  // namespace

vofp_status rbc_ensure(vofp_ctx* c) {
    if (c->rbc_built) return VOFP_OK;
    c->rbc_built = true;
    c->rbc_ok = false;
    const Dims d = c->d;
    // compact tensor maps: N/2 pairs per row, rows of 16-byte multiples (nx multiple of 8);
    // VOFP_RB_COMPACT=0 keeps the interleaved red-black kernel
    const char* env = std::getenv("VOFP_RB_COMPACT");
    if (env && std::strcmp(env, "0") == 0) return VOFP_OK;
    if (!c->tma_ok[0] || d.nx % 8 != 0 || !c->Txf) return VOFP_OK;
    cudaStream_t st = c->stream;
    vofp_status s;
    const long long nh = d.n / 2;
    // scratch: exception flags per cell and chunk counts
    const int nchunks = (int)((d.n + kChunk - 1) / kChunk);
    uint8_t* isexc = reinterpret_cast<uint8_t*>(c->work);            // N doubles of scratch: 2N bytes used
    uint8_t* isgrp = isexc + d.n;
    unsigned int* counts = reinterpret_cast<unsigned int*>(c->partials);
    unsigned int* offsets = counts + nchunks + 1;
    if (2 * (nchunks + 1) > 2 * kMaxPartials) return VOFP_OK;
    // exceptions
    launch(c, k_cmp_count<0>, nchunks, kNT, st, d, (const int32_t*)c->root, (const uint32_t*)c->red_bits,
           (const uint8_t*)nullptr, counts);
    launch(c, k_cmp_scan, 1, 1024, st, nchunks, counts, offsets);
    unsigned int ne = 0;
    VOFP_CUDA_TRY(c, cudaMemcpyAsync(&ne, counts + nchunks, sizeof(ne), cudaMemcpyDeviceToHost, st));
    VOFP_CUDA_TRY(c, cudaStreamSynchronize(st));
    const long long need = nh + ne;
    if (need > c->rbc_cap) {
        // grow (once per operator size class): the compact vectors and per-entry bits
        const long long cap = need + need / 8 + 1024;
        if ((s = c->alloc(&c->rbc_r, cap)) || (s = c->alloc(&c->rbc_p0, cap)) || (s = c->alloc(&c->rbc_p1, cap)) ||
            (s = c->alloc(&c->rbc_x, cap)) || (s = c->alloc(&c->rbc_q, cap)) ||
            (s = c->alloc(&c->rbc_bits, (cap + 31) / 32)) || (s = c->alloc(&c->rbc_exc, cap - nh)) ||
            (s = c->alloc(&c->rbc_fcell, 6 * (cap - nh))) || (s = c->alloc(&c->rbc_fh, 6 * (cap - nh))) ||
            (s = c->alloc(&c->rbc_fexc, 36 * (cap - nh))) || (s = c->alloc(&c->rbc_fT, 36 * (cap - nh))) ||
            (s = c->alloc(&c->rbc_enb, 6 * (cap - nh))) || (s = c->alloc(&c->rbc_eT, 6 * (cap - nh))) ||
            (s = c->alloc(&c->rbc_dE, cap - nh + 1)))
            return s;
        c->rbc_cap = cap;
        for (float* v : {c->rbc_r, c->rbc_p0, c->rbc_p1, c->rbc_x, c->rbc_q})
            VOFP_CUDA_TRY(c, cudaMemsetAsync(v, 0, sizeof(float) * cap, st));
    }
    int ncells = 0;
    if (c->ngroups > 0) {
        VOFP_CUDA_TRY(c, cudaMemcpyAsync(&ncells, c->gptr + c->ngroups, sizeof(int), cudaMemcpyDeviceToHost, st));
        VOFP_CUDA_TRY(c, cudaStreamSynchronize(st));
        if (ncells > d.n / 4) return VOFP_OK;
        if (!c->rbc_gref &&
            ((s = c->alloc(&c->rbc_gref, (long long)d.n / 4 + 1)) || (s = c->alloc(&c->rbc_gfx, (long long)d.n / 4 + 1)) ||
             (s = c->alloc(&c->rbc_gm, 4 * ((long long)d.n / 8 + 1))) ||
             (s = c->alloc(&c->rbc_gf, 4 * ((long long)d.n / 8 + 1))) || (s = c->alloc(&c->rbc_gn, (long long)d.n / 8 + 1))))
            return s;
    }
    launch(c, k_cmp_write<0>, nchunks, kNT, st, d, (const int32_t*)c->root, (const uint32_t*)c->red_bits,
           (const uint8_t*)nullptr, (const unsigned int*)offsets, c->rbc_exc);
    if (ne > 0)
        launch(c, k_exc_tables, ceil_div(ne, kNT), kNT, st, d, (int)ne, (const int*)c->rbc_exc, (const float*)c->Txf,
               (const float*)c->Tyf, (const float*)c->Tzf, c->rbc_enb, c->rbc_eT);
    // rows next to exceptions
    VOFP_CUDA_TRY(c, cudaMemsetAsync(isexc, 0, 2 * d.n, st));
    if (ne > 0) launch(c, k_mark, ceil_div(ne, kNT), kNT, st, (int)ne, (const int*)c->rbc_exc, isexc, (uint8_t)1);
    if (ncells > 0) launch(c, k_mark, ceil_div(ncells, kNT), kNT, st, ncells, (const int*)c->gcells, isgrp, (uint8_t)1);
    launch(c, k_cmp_count<1>, nchunks, kNT, st, d, (const int32_t*)nullptr, (const uint32_t*)nullptr,
           (const uint8_t*)isexc, counts);
    launch(c, k_cmp_scan, 1, 1024, st, nchunks, counts, offsets);
    unsigned int nf = 0;
    VOFP_CUDA_TRY(c, cudaMemcpyAsync(&nf, counts + nchunks, sizeof(nf), cudaMemcpyDeviceToHost, st));
    VOFP_CUDA_TRY(c, cudaStreamSynchronize(st));
    if ((long long)nf + 1 > 6 * (c->rbc_cap - nh)) return VOFP_OK;    // cannot happen: 6 faces per exception
    launch(c, k_cmp_write<1>, nchunks, kNT, st, d, (const int32_t*)nullptr, (const uint32_t*)nullptr,
           (const uint8_t*)isexc, (const unsigned int*)offsets, c->rbc_fcell);
    launch(c, k_fix_faces, ceil_div(nf + 1, kNT), kNT, st, d, (int)nf, (const int*)c->rbc_fcell,
               (const int*)c->rbc_exc, (int)ne, (const uint8_t*)isexc, (const uint8_t*)isgrp, (const float*)c->Txf,
               (const float*)c->Tyf, (const float*)c->Tzf, c->rbc_fexc, c->rbc_fT, c->rbc_fh);
    launch(c, k_cbits, grid_n((need + 31) / 32), kNT, st, d, nh, (int)ne, (const int*)c->rbc_exc,
           (const int32_t*)c->root, c->rbc_bits);
    if (ncells > 0) {
        launch(c, k_gref, ceil_div(ncells, kNT), kNT, st, d, ncells, (const int*)c->gcells, (const int*)c->rbc_exc,
               (int)ne, (const int*)c->rbc_fcell, (int)nf, nh, c->rbc_gref, c->rbc_gfx);
        launch(c, k_gflat, ceil_div(c->ngroups, kNT), kNT, st, c->ngroups, (const int*)c->gptr,
               (const int*)c->rbc_gref, (const int*)c->rbc_gfx, (int)nf, reinterpret_cast<int4*>(c->rbc_gm),
               reinterpret_cast<int4*>(c->rbc_gf), c->rbc_gn);
    }
    // the zero difference entry behind faces without an exception
    VOFP_CUDA_TRY(c, cudaMemsetAsync(c->rbc_dE + ne, 0, sizeof(float), st));
    // rows per thread of the iteration kernel: 2 (32 x 16 tiles) unless VOFP_RBC_ROWS=1 (32 x 8)
    {
        const char* env = std::getenv("VOFP_RBC_ROWS");
        c->rbc_rpt = (env && std::strcmp(env, "1") == 0) ? 1 : 2;
    }
    const int th = kBY * c->rbc_rpt;
    // the iteration kernel's dynamic shared memory and resident blocks
    int nb = 0;
    if (c->rbc_rpt == 1) {
        constexpr size_t smem = cg_rbc_smem<kRbcStages, 1>();
        cudaFuncSetAttribute(k_rbc_tma<kRbcStages, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_rbc_tma<kRbcStages, 1>, kBX * kBY, smem) != cudaSuccess)
            nb = 0;
    } else {
        constexpr size_t smem = cg_rbc_smem<kRbcStages, 2>();
        cudaFuncSetAttribute(k_rbc_tma<kRbcStages, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_rbc_tma<kRbcStages, 2>, kBX * kBY, smem) != cudaSuccess)
            nb = 0;
    }
    cudaGetLastError();
    VOFP_CUDA_TRY(c, cudaStreamSynchronize(st));
    if (nb <= 0) return VOFP_OK;
    {
        const long long tiles_x = ceil_div(d.nx / 2, RbcGeom::NP), tiles_y = ceil_div(d.ny, th);
        // the kernel's work index is an int
        if (tiles_x * tiles_y * (d.nz + 2 * kSegSteps) > 0x7fffffffLL) return VOFP_OK;
        int fgx = 0, fgy = 0;
        if (parse_group(&fgx, &fgy) && (tiles_x % fgx || tiles_y % fgy || (long long)fgx * fgy > kMaxGroup)) fgx = fgy = 0;
        c->rbc_nblocks = 0;
        rbc_split(tiles_x, tiles_y, d.nz, (long long)num_sms() * nb, fgx, fgy, &c->rbc_split, &c->rbc_nblocks);
        if (c->rbc_nblocks <= 0) return VOFP_OK;
        const int ng = c->ngroups;
        if (c->rbc_nblocks + ceil_div(nf + ng, (long long)kNT) > kMaxPartials / 4 - 16) return VOFP_OK;
    }
    c->rbc_blocks_per_sm = nb;
    c->rbc_nh = nh;
    c->rbc_ne = (int)ne;
    c->rbc_nf = (int)nf;
    c->rbc_ok = true;
    return VOFP_OK;
}

void rbc_prep(vofp_ctx* c, cudaStream_t st, const double* rhs) {
    const long long nc = c->rbc_nh + c->rbc_ne;
    launch(c, k_rbc_prep, grid_n(nc), kNT, st, c->d, c->rbc_nh, c->rbc_ne, (const int*)c->rbc_exc, rhs,
           (const uint32_t*)c->rbc_bits, c->rbc_r, c->rbc_x, c->rbc_p0, c->sc, c->partials, c->counters);
}

namespace {
template <int RPT>
void launch_main_t(vofp_ctx* c, cudaStream_t st, const float* po, float* pn, bool pdl) {
    using G = RbcGeomT<RPT>;
    const Dims d = c->d;
    const int nh = d.nx / 2;
    const CUtensorMap *mr = tensor_map_f32_x(c, c->rbc_r, nh, G::BWC, G::TH + 4),
                      *mp = tensor_map_f32_x(c, po, nh, G::BWC, G::TH + 4),
                      *mx = tensor_map_f32(c, c->Txf, G::BWF, G::TH + 2),
                      *my = tensor_map_f32(c, c->Tyf, G::BWF, G::TH + 3),
                      *mz = tensor_map_f32(c, c->Tzf, G::BWF, G::TH + 2);
    if (!(mr && mp && mx && my && mz)) {
        c->set_error("tensor map of the compact red-black vectors could not be built");
        return;
    }
    RbcMaps maps;
    maps.r = *mr;
    maps.p = *mp;
    maps.tx = *mx;
    maps.ty = *my;
    maps.tz = *mz;
    const RbcExc ex{(const float*)c->rbc_r, (const int*)c->rbc_enb, (const float*)c->rbc_eT, c->rbc_dE,
                    c->rbc_nh, c->rbc_ne};
    launch_dep(c, pdl, k_rbc_tma<kRbcStages, RPT>, dim3(c->rbc_nblocks), dim3(kBX, kBY),
               cg_rbc_smem<kRbcStages, RPT>(), st, maps, d, c->rbc_split, ex, po, pn, c->rbc_x, c->rbc_q,
               c->sc, c->partials + kPqBase);
}
void launch_main(vofp_ctx* c, cudaStream_t st, const float* po, float* pn, bool pdl) {
    if (c->rbc_rpt == 1)
        launch_main_t<1>(c, st, po, pn, pdl);
    else
        launch_main_t<2>(c, st, po, pn, pdl);
}
}  // namespace

// the rows next to exceptions and the merge groups (the exception rows are formed in the
// iteration kernel)
void rbc_aux(vofp_ctx* c, cudaStream_t st, const float* po, float* pn, bool pdl) {
    (void)po;
    const int ng = c->rbc_gm ? c->ngroups : 0;
    if (c->rbc_nf + ng > 0)
        launch_dep(c, pdl, k_rbc_fix_rows, dim3(ceil_div(c->rbc_nf + ng, kNT)), dim3(kNT), 0, st, c->rbc_nf, ng,
                   (const int*)c->rbc_fh, (const int*)c->rbc_fexc, (const float*)c->rbc_fT, (const float*)c->rbc_dE,
                   (const int4*)c->rbc_gm, (const int4*)c->rbc_gf, (const int*)c->rbc_gn, (const int*)c->gptr,
                   (const int*)c->rbc_gref, (const int*)c->rbc_gfx, (const double*)c->gcorr, (const float*)pn,
                   c->rbc_q, c->partials + kPqBase + c->rbc_nblocks);
}

// block partials of p.Ap that the iteration kernel and the fix rows leave for the update
int rbc_pq_parts(const vofp_ctx* c) {
    const int ng = c->rbc_gm ? c->ngroups : 0;
    return c->rbc_nblocks + (c->rbc_nf + ng > 0 ? ceil_div(c->rbc_nf + ng, kNT) : 0);
}

void rbc_iteration(vofp_ctx* c, cudaStream_t st, const float* po, float* pn, cudaGraphConditionalHandle h,
                   int use_h) {
    // In the solve's graph (use_h set; a refused launch is caught when the capture ends) the three
    // kernels of an iteration (iteration kernel with the exception rows, fix rows, update), and
    // the next iteration's first, are chained by programmatic dependent launch: each waits for its
    // predecessor before it reads, so only the launch latency and the block set-up overlap the
    // predecessor's drain. The short fix kernel releases its successor's blocks at once; the
    // iteration kernel and the update release theirs as their own blocks end (blocks of the next
    // kernel resident early beside the streaming ones slowed the solve: 395.2 ms with every kernel
    // releasing early, 387.8 ms with the update also releasing, 386.2 ms with the short kernels
    // only, 388.2 ms without the chaining, measured with a separate exception kernel). The
    // host-driven loop launches them as ordinary kernels.
    const bool pdl = c->pdl != 0 && use_h != 0;
    launch_main(c, st, po, pn, pdl);
    rbc_aux(c, st, po, pn, pdl);
    const long long nc = c->rbc_nh + c->rbc_ne;
    // the update: one wave of four 256-thread blocks per SM (its register cap); two waves of eight
    // per SM took 7.5 us more per iteration at 512x256x128
    const int ug = std::min(grid_n(nc / 4 + 1), num_sms() * 4);
    launch_dep(c, pdl, k_cg_update<float, true>, dim3(ug), dim3(kNT), 0, st, nc, c->rbc_r,
               (const float*)c->rbc_q, (const uint32_t*)c->rbc_bits, c->sc, c->partials, c->counters, h, use_h,
               (const double*)(c->partials + kPqBase), rbc_pq_parts(c));
}

void rbc_finish_xf(vofp_ctx* c, cudaStream_t st) {
    launch(c, k_rbc_expand, grid_n(c->d.n), kNT, st, c->d, (const float*)c->rbc_x, (const float*)c->rbc_p0, c->xf,
           (const CgScalars*)c->sc);
    if (c->rbc_ne > 0)
        launch(c, k_rbc_expand_exc, ceil_div(c->rbc_ne, kNT), kNT, st, c->rbc_nh, c->rbc_ne, (const int*)c->rbc_exc,
               (const float*)c->rbc_x, (const float*)c->rbc_p0, c->xf, (const CgScalars*)c->sc);
}

// timed as ordinary launches, one kernel after the other
void rbc_time_kernel(vofp_ctx* c, cudaStream_t st) { launch_main(c, st, c->rbc_p0, c->rbc_p1, false); }
void rbc_time_aux(vofp_ctx* c, cudaStream_t st) { rbc_aux(c, st, c->rbc_p0, c->rbc_p1, false); }

}  // namespace vofp

extern "C" vofp_status vofp_rbc_split_plan(int tiles_x, int tiles_y, int nz, int slots, int* blocks, int* per,
                                           int* pad, int* gx, int* gy) {
    if (tiles_x <= 0 || tiles_y <= 0 || nz <= 0 || slots <= 0 || !blocks || !per || !pad || !gx || !gy)
        return VOFP_ERR_INVALID_ARG;
    if ((long long)tiles_x * tiles_y * (nz + 2 * vofp::kSegSteps) > 0x7fffffffLL) return VOFP_ERR_INVALID_ARG;
    vofp::RbcSplit sp{};
    int nb = 0;
    vofp::rbc_split(tiles_x, tiles_y, nz, slots, 0, 0, &sp, &nb);
    *blocks = nb;
    *per = sp.per;
    *pad = sp.pad;
    *gx = sp.gx;
    *gy = sp.gy;
    return VOFP_OK;
}
