// Operator assembly of the pressure Poisson equation (Sec. 2 Eq. density; Sec. 2.3 Eqs.
// integral1-integral2 and cell merging; Sec. 2.10 density smoothing) and the divergence
// right-hand side (Sec. 2.1 Eq. poisson1; Sec. 2.4 F_i = A_i u_i).
//
// Cell-centred kernels: each thread owns one cell and writes the coefficient of its +x, +y and
// +z face, so every face coefficient is computed once and stored once (structure of arrays).
#include <algorithm>
#include <cmath>

#include "vofp_internal.cuh"

namespace vofp {
namespace {

constexpr int kNT = 256;


// rho = rho_g + (rho_l - rho_g) F   (Eq. density with H(phi) = phi)
__global__ void k_density(Dims d, const double* __restrict__ F, double rl, double rg,
                          double* __restrict__ rho) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < d.n;
         c += (long long)gridDim.x * blockDim.x)
        rho[c] = rg + (rl - rg) * F[c];
}

// one pass of the (1/4, 1/2, 1/4) filter along `axis` (0 = x, 1 = y, 2 = z); a missing
// neighbour at a domain wall is replaced by the cell itself (Sec. 2.10)
__global__ void k_smooth(Dims d, int axis, const double* __restrict__ in, double* __restrict__ out) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < d.n;
         c += (long long)gridDim.x * blockDim.x) {
        int i, j, k;
        cell_ijk(d, c, i, j, k);
        long long st = axis == 0 ? 1 : axis == 1 ? d.nx : d.plane;
        int pos = axis == 0 ? i : axis == 1 ? j : k;
        int len = axis == 0 ? d.nx : axis == 1 ? d.ny : d.nz;
        double lo = pos > 0 ? in[c - st] : in[c];
        double hi = pos < len - 1 ? in[c + st] : in[c];
        out[c] = 0.25 * lo + 0.5 * in[c] + 0.25 * hi;
    }
}

__global__ void k_activity_init(Dims d, const double* __restrict__ vf, uint8_t* __restrict__ ina) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < d.n;
         c += (long long)gridDim.x * blockDim.x)
        ina[c] = vf ? (uint8_t)!(vf[c] > 0.0) : (uint8_t)0;
}

struct Bc6 {
    int k[6];
};

// A cell loses its unknown when none of its flux-carrying faces (interior faces towards a cell
// that still has one, or p = 0 domain faces) is open.
__global__ void k_activity_step(Dims d, Bc6 bc, const double* __restrict__ ax,
                                const double* __restrict__ ay, const double* __restrict__ az,
                                const uint8_t* __restrict__ in, uint8_t* __restrict__ out,
                                unsigned int* changed) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < d.n;
         c += (long long)gridDim.x * blockDim.x) {
        if (in[c]) {
            out[c] = 1;
            continue;
        }
        int i, j, k;
        cell_ijk(d, c, i, j, k);
        bool open = false;
        open |= ax[fx_idx(d, i, j, k)] > 0.0 && (i > 0 ? !in[c - 1] : bc.k[0] == VOFP_BC_DIRICHLET);
        open |= ax[fx_idx(d, i + 1, j, k)] > 0.0 && (i < d.nx - 1 ? !in[c + 1] : bc.k[1] == VOFP_BC_DIRICHLET);
        open |= ay[fy_idx(d, i, j, k)] > 0.0 && (j > 0 ? !in[c - d.nx] : bc.k[2] == VOFP_BC_DIRICHLET);
        open |= ay[fy_idx(d, i, j + 1, k)] > 0.0 && (j < d.ny - 1 ? !in[c + d.nx] : bc.k[3] == VOFP_BC_DIRICHLET);
        open |= az[fz_idx(d, i, j, k)] > 0.0 && (k > 0 ? !in[c - d.plane] : bc.k[4] == VOFP_BC_DIRICHLET);
        open |= az[fz_idx(d, i, j, k + 1)] > 0.0 && (k < d.nz - 1 ? !in[c + d.plane] : bc.k[5] == VOFP_BC_DIRICHLET);
        out[c] = open ? 0 : 1;
        if (!open) atomicAdd(changed, 1u);
    }
}

// effective apertures: faces touching a cell without an unknown are closed
__global__ void k_eff_apertures(Dims d, const double* __restrict__ ax, const double* __restrict__ ay,
                                const double* __restrict__ az, const uint8_t* __restrict__ ina,
                                double* __restrict__ axe, double* __restrict__ aye,
                                double* __restrict__ aze) {
    const long long nfx = (long long)(d.nx + 1) * d.ny * d.nz;
    const long long nfy = (long long)d.nx * (d.ny + 1) * d.nz;
    const long long nfz = (long long)d.nx * d.ny * (d.nz + 1);
    for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < nfx + nfy + nfz;
         f += (long long)gridDim.x * blockDim.x) {
        if (f < nfx) {
            int i = int(f % (d.nx + 1));
            long long t = f / (d.nx + 1);
            long long c = i + d.nx * t;   // cell to the right of face i (row t)
            bool okl = i == 0 || !ina[c - 1];
            bool okr = i == d.nx || !ina[c];
            axe[f] = (okl && okr) ? ax[f] : 0.0;
        } else if (f < nfx + nfy) {
            long long g = f - nfx;
            int i = int(g % d.nx);
            long long t = g / d.nx;
            int j = int(t % (d.ny + 1));
            int k = int(t / (d.ny + 1));
            long long c = i + d.nx * (j + (long long)d.ny * k);
            bool okl = j == 0 || !ina[c - d.nx];
            bool okr = j == d.ny || !ina[c];
            aye[g] = (okl && okr) ? ay[g] : 0.0;
        } else {
            long long g = f - nfx - nfy;
            long long plane = d.plane;
            int k = int(g / plane);
            long long c = g;   // cell above face k has the same in-plane index at layer k
            bool okl = k == 0 || !ina[c - plane];
            bool okr = k == d.nz || !ina[c];
            aze[g] = (okl && okr) ? az[g] : 0.0;
        }
    }
}

// T of each cell's +x, +y, +z face: A_f S_f / ((d_L rho_L + d_R rho_R) / 2); 0 on domain faces
// T of each cell's +x, +y, +z interior face, and the face's inverse resistance
// kappa = 1 / ((d_L rho_L + d_R rho_R) / 2) where the face is open (0 where it is closed or on the
// domain boundary), which the projection of the face velocities uses
__global__ void k_face_coeffs(Dims d, const double* __restrict__ dx, const double* __restrict__ dy,
                              const double* __restrict__ dz, const double* __restrict__ rho,
                              const double* __restrict__ axe, const double* __restrict__ aye,
                              const double* __restrict__ aze, double* __restrict__ Tx,
                              double* __restrict__ Ty, double* __restrict__ Tz, double* __restrict__ kx,
                              double* __restrict__ ky, double* __restrict__ kz) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < d.n;
         c += (long long)gridDim.x * blockDim.x) {
        int i, j, k;
        cell_ijk(d, c, i, j, k);
        const double rc = rho[c];
        double tx = 0.0, ty = 0.0, tz = 0.0, qx = 0.0, qy = 0.0, qz = 0.0;
        // one FP64 division per face (the FP64 pipe bounds this kernel): T = (A S) (1 / den)
        if (i < d.nx - 1) {
            const double a = axe[fx_idx(d, i + 1, j, k)], inv = 1.0 / (0.5 * (dx[i] * rc + dx[i + 1] * rho[c + 1]));
            tx = (a * (dz[k] * dy[j])) * inv;
            qx = a > 0.0 ? inv : 0.0;
        }
        if (j < d.ny - 1) {
            const double a = aye[fy_idx(d, i, j + 1, k)], inv = 1.0 / (0.5 * (dy[j] * rc + dy[j + 1] * rho[c + d.nx]));
            ty = (a * (dz[k] * dx[i])) * inv;
            qy = a > 0.0 ? inv : 0.0;
        }
        if (k < d.nz - 1) {
            const double a = aze[fz_idx(d, i, j, k + 1)], inv = 1.0 / (0.5 * (dz[k] * rc + dz[k + 1] * rho[c + d.plane]));
            tz = (a * (dy[j] * dx[i])) * inv;
            qz = a > 0.0 ? inv : 0.0;
        }
        Tx[c] = tx;
        Ty[c] = ty;
        Tz[c] = tz;
        kx[c] = qx;
        ky[c] = qy;
        kz[c] = qz;
    }
}

// The same two kernels on x-pairs of cells (nx even): a thread takes cells c and c + 1 of one row
// (c even, so every cell-indexed and y/z-face stream is 16-byte aligned) and moves the
// structure-of-arrays streams as double2 words; the x-face apertures (rows of nx + 1) stay
// scalar.  Each cell's arithmetic is that of the scalar kernels, operation for operation.
__device__ __forceinline__ double2 ld2(const double* __restrict__ p, long long c) {
    return *reinterpret_cast<const double2*>(p + c);
}
__device__ __forceinline__ void st2(double* __restrict__ p, long long c, double a, double b) {
    *reinterpret_cast<double2*>(p + c) = make_double2(a, b);
}
__global__ void k_face_coeffs2(Dims d, const double* __restrict__ dx, const double* __restrict__ dy,
                               const double* __restrict__ dz, const double* __restrict__ rho,
                               const double* __restrict__ axe, const double* __restrict__ aye,
                               const double* __restrict__ aze, double* __restrict__ Tx,
                               double* __restrict__ Ty, double* __restrict__ Tz, double* __restrict__ kx,
                               double* __restrict__ ky, double* __restrict__ kz) {
    const long long npairs = d.n / 2;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < npairs;
         q += (long long)gridDim.x * blockDim.x) {
        const long long c = 2 * q;
        int i, j, k;
        cell_ijk(d, c, i, j, k);
        const double2 r2 = ld2(rho, c);
        const double rc[2] = {r2.x, r2.y};
        double tx[2] = {0.0, 0.0}, ty[2] = {0.0, 0.0}, tz[2] = {0.0, 0.0};
        double qx[2] = {0.0, 0.0}, qy[2] = {0.0, 0.0}, qz[2] = {0.0, 0.0};
        // +x faces: cell c's is interior (i + 1 < nx), cell c + 1's when i + 2 < nx
        {
            const double a0 = axe[fx_idx(d, i + 1, j, k)];
            const double inv0 = 1.0 / (0.5 * (dx[i] * rc[0] + dx[i + 1] * rc[1]));
            tx[0] = (a0 * (dz[k] * dy[j])) * inv0;
            qx[0] = a0 > 0.0 ? inv0 : 0.0;
            if (i + 1 < d.nx - 1) {
                const double a1 = axe[fx_idx(d, i + 2, j, k)];
                const double inv1 = 1.0 / (0.5 * (dx[i + 1] * rc[1] + dx[i + 2] * rho[c + 2]));
                tx[1] = (a1 * (dz[k] * dy[j])) * inv1;
                qx[1] = a1 > 0.0 ? inv1 : 0.0;
            }
        }
        if (j < d.ny - 1) {
            const double2 a = ld2(aye, fy_idx(d, i, j + 1, k)), rn = ld2(rho, c + d.nx);
            const double av[2] = {a.x, a.y}, rv[2] = {rn.x, rn.y};
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const double inv = 1.0 / (0.5 * (dy[j] * rc[e] + dy[j + 1] * rv[e]));
                ty[e] = (av[e] * (dz[k] * dx[i + e])) * inv;
                qy[e] = av[e] > 0.0 ? inv : 0.0;
            }
        }
        if (k < d.nz - 1) {
            const double2 a = ld2(aze, fz_idx(d, i, j, k + 1)), rn = ld2(rho, c + d.plane);
            const double av[2] = {a.x, a.y}, rv[2] = {rn.x, rn.y};
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const double inv = 1.0 / (0.5 * (dz[k] * rc[e] + dz[k + 1] * rv[e]));
                tz[e] = (av[e] * (dy[j] * dx[i + e])) * inv;
                qz[e] = av[e] > 0.0 ? inv : 0.0;
            }
        }
        st2(Tx, c, tx[0], tx[1]);
        st2(Ty, c, ty[0], ty[1]);
        st2(Tz, c, tz[0], tz[1]);
        st2(kx, c, qx[0], qx[1]);
        st2(ky, c, qy[0], qy[1]);
        st2(kz, c, qz[0], qz[1]);
    }
}

__global__ void k_diag2(Dims d, Bc6 bc, const double* __restrict__ dx, const double* __restrict__ dy,
                        const double* __restrict__ dz, const double* __restrict__ rho,
                        const double* __restrict__ axe, const double* __restrict__ aye,
                        const double* __restrict__ aze, const double* __restrict__ Tx,
                        const double* __restrict__ Ty, const double* __restrict__ Tz, double* __restrict__ diag) {
    const long long npairs = d.n / 2;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < npairs;
         q += (long long)gridDim.x * blockDim.x) {
        const long long c = 2 * q;
        int i, j, k;
        cell_ijk(d, c, i, j, k);
        const double2 x2 = ld2(Tx, c), y2 = ld2(Ty, c), z2 = ld2(Tz, c), r2 = ld2(rho, c);
        const double2 ym = j > 0 ? ld2(Ty, c - d.nx) : make_double2(0.0, 0.0);
        const double2 zm = k > 0 ? ld2(Tz, c - d.plane) : make_double2(0.0, 0.0);
        const double txs[2] = {x2.x, x2.y}, tys[2] = {y2.x, y2.y}, tzs[2] = {z2.x, z2.y}, rcs[2] = {r2.x, r2.y};
        const double tym[2] = {ym.x, ym.y}, tzm[2] = {zm.x, zm.y};
        const double txm[2] = {i > 0 ? Tx[c - 1] : 0.0, x2.x};
        double out[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int ii = i + e;
            const double rc = rcs[e];
            double s = txs[e] + tys[e] + tzs[e];
            if (ii > 0) s += txm[e];
            if (j > 0) s += tym[e];
            if (k > 0) s += tzm[e];
            if (ii == 0 && bc.k[0] == VOFP_BC_DIRICHLET) s += (axe[fx_idx(d, 0, j, k)] * (dz[k] * dy[j])) / (0.5 * dx[0] * rc);
            if (ii == d.nx - 1 && bc.k[1] == VOFP_BC_DIRICHLET) s += (axe[fx_idx(d, d.nx, j, k)] * (dz[k] * dy[j])) / (0.5 * dx[ii] * rc);
            if (j == 0 && bc.k[2] == VOFP_BC_DIRICHLET) s += (aye[fy_idx(d, ii, 0, k)] * (dz[k] * dx[ii])) / (0.5 * dy[0] * rc);
            if (j == d.ny - 1 && bc.k[3] == VOFP_BC_DIRICHLET) s += (aye[fy_idx(d, ii, d.ny, k)] * (dz[k] * dx[ii])) / (0.5 * dy[j] * rc);
            if (k == 0 && bc.k[4] == VOFP_BC_DIRICHLET) s += (aze[fz_idx(d, ii, j, 0)] * (dy[j] * dx[ii])) / (0.5 * dz[0] * rc);
            if (k == d.nz - 1 && bc.k[5] == VOFP_BC_DIRICHLET) s += (aze[fz_idx(d, ii, j, d.nz)] * (dy[j] * dx[ii])) / (0.5 * dz[k] * rc);
            out[e] = s;
        }
        st2(diag, c, out[0], out[1]);
    }
}

// diagonal of the unmerged operator: sum of the six face coefficients plus p = 0 faces
__global__ void k_diag(Dims d, Bc6 bc, const double* __restrict__ dx, const double* __restrict__ dy,
                       const double* __restrict__ dz, const double* __restrict__ rho,
                       const double* __restrict__ axe, const double* __restrict__ aye,
                       const double* __restrict__ aze, const double* __restrict__ Tx,
                       const double* __restrict__ Ty, const double* __restrict__ Tz,
                       double* __restrict__ diag) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < d.n;
         c += (long long)gridDim.x * blockDim.x) {
        int i, j, k;
        cell_ijk(d, c, i, j, k);
        const double rc = rho[c];
        double s = Tx[c] + Ty[c] + Tz[c];
        if (i > 0) s += Tx[c - 1];
        if (j > 0) s += Ty[c - d.nx];
        if (k > 0) s += Tz[c - d.plane];
        if (i == 0 && bc.k[0] == VOFP_BC_DIRICHLET) s += (axe[fx_idx(d, 0, j, k)] * (dz[k] * dy[j])) / (0.5 * dx[0] * rc);
        if (i == d.nx - 1 && bc.k[1] == VOFP_BC_DIRICHLET) s += (axe[fx_idx(d, d.nx, j, k)] * (dz[k] * dy[j])) / (0.5 * dx[i] * rc);
        if (j == 0 && bc.k[2] == VOFP_BC_DIRICHLET) s += (aye[fy_idx(d, i, 0, k)] * (dz[k] * dx[i])) / (0.5 * dy[0] * rc);
        if (j == d.ny - 1 && bc.k[3] == VOFP_BC_DIRICHLET) s += (aye[fy_idx(d, i, d.ny, k)] * (dz[k] * dx[i])) / (0.5 * dy[j] * rc);
        if (k == 0 && bc.k[4] == VOFP_BC_DIRICHLET) s += (aze[fz_idx(d, i, j, 0)] * (dy[j] * dx[i])) / (0.5 * dz[0] * rc);
        if (k == d.nz - 1 && bc.k[5] == VOFP_BC_DIRICHLET) s += (aze[fz_idx(d, i, j, d.nz)] * (dy[j] * dx[i])) / (0.5 * dz[k] * rc);
        diag[c] = s;
    }
}

// Cells with an unknown and open volume below the threshold: their merge target is the neighbour
// across the interior face of largest open area (first of -x,+x,-y,+y,-z,+z on ties).
// Pass 0 counts, pass 1 writes (cell, target) pairs (order of the list is not significant).
__global__ void k_small_cells(Dims d, double thr, const double* __restrict__ vf,
                              const uint8_t* __restrict__ ina, const double* __restrict__ dx,
                              const double* __restrict__ dy, const double* __restrict__ dz,
                              const double* __restrict__ axe, const double* __restrict__ aye,
                              const double* __restrict__ aze, unsigned int* count, long long cap,
                              long long* __restrict__ cells, long long* __restrict__ targets,
                              double* __restrict__ vfs) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < d.n;
         c += (long long)gridDim.x * blockDim.x) {
        if (ina[c] || !(vf[c] < thr)) continue;
        int i, j, k;
        cell_ijk(d, c, i, j, k);
        double a[6];
        a[0] = i > 0 ? axe[fx_idx(d, i, j, k)] * (dz[k] * dy[j]) : 0.0;
        a[1] = i < d.nx - 1 ? axe[fx_idx(d, i + 1, j, k)] * (dz[k] * dy[j]) : 0.0;
        a[2] = j > 0 ? aye[fy_idx(d, i, j, k)] * (dz[k] * dx[i]) : 0.0;
        a[3] = j < d.ny - 1 ? aye[fy_idx(d, i, j + 1, k)] * (dz[k] * dx[i]) : 0.0;
        a[4] = k > 0 ? aze[fz_idx(d, i, j, k)] * (dy[j] * dx[i]) : 0.0;
        a[5] = k < d.nz - 1 ? aze[fz_idx(d, i, j, k + 1)] * (dy[j] * dx[i]) : 0.0;
        int best = 0;
        for (int f = 1; f < 6; ++f)
            if (a[f] > a[best]) best = f;
        if (!(a[best] > 0.0)) continue;
        const long long off[6] = {-1, 1, -(long long)d.nx, (long long)d.nx, -d.plane, d.plane};
        // slots in arrival order; the caller grows the lists and runs again if they overflow
        const unsigned int slot = atomicAdd(count, 1u);
        if ((long long)slot < cap) {
            cells[slot] = c;
            targets[slot] = c + off[best];
            vfs[slot] = vf[c];
        }
    }
}

// slot_of[cell] = slot of every listed small cell (the other entries were set to -1 before)
__global__ void k_small_slots(int m, const long long* __restrict__ cells, int32_t* __restrict__ slot_of) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < m) slot_of[cells[t]] = t;
}

// slot of each small cell's target among the small cells, -1 if the target is not one of them
__global__ void k_small_target_slots(int m, const long long* __restrict__ targets,
                                     const int32_t* __restrict__ slot_of, int32_t* __restrict__ tslot) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < m) tslot[t] = slot_of[targets[t]];
}

__global__ void k_count_u8(long long n, const uint8_t* __restrict__ a, unsigned int* count) {
    unsigned int local = 0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x)
        local += a[c] ? 1u : 0u;
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(count, local);
}

__global__ void k_root_init(Dims d, const uint8_t* __restrict__ ina, int32_t* __restrict__ root) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < d.n;
         c += (long long)gridDim.x * blockDim.x)
        root[c] = ina[c] ? -1 : (int32_t)c;
}

__global__ void k_root_scatter(int m, const long long* __restrict__ cells,
                               const long long* __restrict__ roots, int32_t* __restrict__ root) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < m) root[cells[t]] = (int32_t)roots[t];
}

__global__ void k_scale_cells(Dims d, const uint8_t* __restrict__ ina, const double* __restrict__ diag,
                              double* __restrict__ s, double* __restrict__ sq) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < d.n;
         c += (long long)gridDim.x * blockDim.x) {
        if (ina[c]) {
            s[c] = 0.0;
            sq[c] = 0.0;
        } else {
            double r = sqrt(diag[c]);
            sq[c] = r;
            s[c] = 1.0 / r;
        }
    }
}

// diag(A_hat) of a merge group = sum over its cells of the diagonal minus the couplings between
// its own cells (both directions); all cells of the group get the group's scale.
__global__ void k_scale_groups(Dims d, int ng, const int* __restrict__ gptr,
                               const int* __restrict__ gcells, const int32_t* __restrict__ root,
                               const double* __restrict__ diag, const double* __restrict__ Tx,
                               const double* __restrict__ Ty, const double* __restrict__ Tz,
                               double* __restrict__ s, double* __restrict__ sq,
                               double* __restrict__ gcorr) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ng) return;
    const int b = gptr[g], e = gptr[g + 1];
    const int32_t m = gcells[b];
    double dsum = 0.0, intra = 0.0;
    for (int t = b; t < e; ++t) {
        long long c = gcells[t];
        int i, j, k;
        cell_ijk(d, c, i, j, k);
        dsum += diag[c];
        if (i > 0 && root[c - 1] == m) intra += Tx[c - 1];
        if (i < d.nx - 1 && root[c + 1] == m) intra += Tx[c];
        if (j > 0 && root[c - d.nx] == m) intra += Ty[c - d.nx];
        if (j < d.ny - 1 && root[c + d.nx] == m) intra += Ty[c];
        if (k > 0 && root[c - d.plane] == m) intra += Tz[c - d.plane];
        if (k < d.nz - 1 && root[c + d.plane] == m) intra += Tz[c];
    }
    const double dhat = dsum - intra;
    const double r = sqrt(dhat);
    const double sm = 1.0 / r;
    for (int t = b; t < e; ++t) {
        s[gcells[t]] = sm;
        sq[gcells[t]] = r;
    }
    gcorr[g] = sm * sm * dsum - double(e - b);
}

__global__ void k_scaled_coeffs(Dims d, const double* __restrict__ s, const double* __restrict__ Tx,
                                const double* __restrict__ Ty, const double* __restrict__ Tz,
                                double* __restrict__ Txs, double* __restrict__ Tys,
                                double* __restrict__ Tzs, float* __restrict__ Txf,
                                float* __restrict__ Tyf, float* __restrict__ Tzf) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < d.n;
         c += (long long)gridDim.x * blockDim.x) {
        int i, j, k;
        cell_ijk(d, c, i, j, k);
        const double sc = s[c];
        double a = i < d.nx - 1 ? sc * Tx[c] * s[c + 1] : 0.0;
        double b = j < d.ny - 1 ? sc * Ty[c] * s[c + d.nx] : 0.0;
        double e = k < d.nz - 1 ? sc * Tz[c] * s[c + d.plane] : 0.0;
        Txs[c] = a;
        Tys[c] = b;
        Tzs[c] = e;
        Txf[c] = (float)a;
        Tyf[c] = (float)b;
        Tzf[c] = (float)e;
    }
}

__global__ void k_slave_bits(Dims d, const int32_t* __restrict__ root, uint32_t* __restrict__ bits) {
    const long long nw = (d.n + 31) / 32;
    for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < nw;
         w += (long long)gridDim.x * blockDim.x) {
        uint32_t v = 0;
        for (int b = 0; b < 32; ++b) {
            long long c = w * 32 + b;
            if (c < d.n && root[c] >= 0 && root[c] != (int32_t)c) v |= (1u << b);
        }
        bits[w] = v;
    }
}

// red cells: (i+j+k) even, own root, and not the master of a multi-cell group (a master always
// touches one of its members, so a neighbour whose root is c marks c as a master)
// Tzr = Tzf with the sign bit set on red cells (coefficients are >= 0, so the sign carries the red
// flag through the same tensor copy as the coefficient; -0.0 marks a red cell with a closed face)
__global__ void k_signed_tz(long long n, const float* __restrict__ tz, const uint32_t* __restrict__ red,
                            float* __restrict__ tzr) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
        tzr[c] = ((red[c >> 5] >> (c & 31)) & 1u) ? -fabsf(tz[c]) : tz[c];
}

__global__ void k_red_bits(Dims d, const int32_t* __restrict__ root, const uint32_t* __restrict__ slave,
                           uint32_t* __restrict__ red, uint32_t* __restrict__ excl, unsigned int* count) {
    const long long nw = (d.n + 31) / 32;
    for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < nw;
         w += (long long)gridDim.x * blockDim.x) {
        uint32_t v = 0;
        for (int b = 0; b < 32; ++b) {
            const long long c = w * 32 + b;
            if (c >= d.n || root[c] != (int32_t)c) continue;
            int i, j, k;
            cell_ijk(d, c, i, j, k);
            if (((i + j + k) & 1) != 0) continue;
            bool master = false;
            if (i > 0) master |= root[c - 1] == (int32_t)c;
            if (i < d.nx - 1) master |= root[c + 1] == (int32_t)c;
            if (j > 0) master |= root[c - d.nx] == (int32_t)c;
            if (j < d.ny - 1) master |= root[c + d.nx] == (int32_t)c;
            if (k > 0) master |= root[c - d.plane] == (int32_t)c;
            if (k < d.nz - 1) master |= root[c + d.plane] == (int32_t)c;
            if (!master) v |= (1u << b);
        }
        red[w] = v;
        excl[w] = v | slave[w];
        if (v) atomicAdd(count, (unsigned int)__popc(v));
    }
}

struct Flux6 {
    const double* g[6];
};

// b_c = -(1/dt) (sum of outward open-face fluxes + body flux) + prescribed Neumann fluxes
__global__ void k_rhs(Dims d, Bc6 bc, Flux6 nf, double dt, const double* __restrict__ dx,
                      const double* __restrict__ dy, const double* __restrict__ dz,
                      const double* __restrict__ axe, const double* __restrict__ aye,
                      const double* __restrict__ aze, const uint8_t* __restrict__ ina,
                      const double* __restrict__ u, const double* __restrict__ v,
                      const double* __restrict__ w, const double* __restrict__ body,
                      double* __restrict__ b) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < d.n;
         c += (long long)gridDim.x * blockDim.x) {
        if (ina[c]) {
            b[c] = 0.0;
            continue;
        }
        int i, j, k;
        cell_ijk(d, c, i, j, k);
        const double Sx = dz[k] * dy[j], Sy = dz[k] * dx[i], Sz = dy[j] * dx[i];
        long long f;
        f = fx_idx(d, i, j, k);
        double fxm = (i == 0 && bc.k[0] != VOFP_BC_DIRICHLET) ? 0.0 : axe[f] * Sx * u[f];
        f = fx_idx(d, i + 1, j, k);
        double fxp = (i == d.nx - 1 && bc.k[1] != VOFP_BC_DIRICHLET) ? 0.0 : axe[f] * Sx * u[f];
        f = fy_idx(d, i, j, k);
        double fym = (j == 0 && bc.k[2] != VOFP_BC_DIRICHLET) ? 0.0 : aye[f] * Sy * v[f];
        f = fy_idx(d, i, j + 1, k);
        double fyp = (j == d.ny - 1 && bc.k[3] != VOFP_BC_DIRICHLET) ? 0.0 : aye[f] * Sy * v[f];
        f = fz_idx(d, i, j, k);
        double fzm = (k == 0 && bc.k[4] != VOFP_BC_DIRICHLET) ? 0.0 : aze[f] * Sz * w[f];
        f = fz_idx(d, i, j, k + 1);
        double fzp = (k == d.nz - 1 && bc.k[5] != VOFP_BC_DIRICHLET) ? 0.0 : aze[f] * Sz * w[f];
        double div = ((fxp - fxm) + (fyp - fym)) + (fzp - fzm);
        if (body) div += body[c];
        double bb = -div / dt;
        if (i == 0 && bc.k[0] == VOFP_BC_NEUMANN && nf.g[0]) bb += axe[fx_idx(d, 0, j, k)] * Sx * nf.g[0][j + (long long)d.ny * k];
        if (i == d.nx - 1 && bc.k[1] == VOFP_BC_NEUMANN && nf.g[1]) bb += axe[fx_idx(d, d.nx, j, k)] * Sx * nf.g[1][j + (long long)d.ny * k];
        if (j == 0 && bc.k[2] == VOFP_BC_NEUMANN && nf.g[2]) bb += aye[fy_idx(d, i, 0, k)] * Sy * nf.g[2][i + (long long)d.nx * k];
        if (j == d.ny - 1 && bc.k[3] == VOFP_BC_NEUMANN && nf.g[3]) bb += aye[fy_idx(d, i, d.ny, k)] * Sy * nf.g[3][i + (long long)d.nx * k];
        if (k == 0 && bc.k[4] == VOFP_BC_NEUMANN && nf.g[4]) bb += aze[fz_idx(d, i, j, 0)] * Sz * nf.g[4][i + (long long)d.nx * j];
        if (k == d.nz - 1 && bc.k[5] == VOFP_BC_NEUMANN && nf.g[5]) bb += aze[fz_idx(d, i, j, d.nz)] * Sz * nf.g[5][i + (long long)d.nx * j];
        b[c] = bb;
    }
}

__global__ void k_group_expand(int ng, const int* __restrict__ gptr, const int* __restrict__ gcells,
                               double* __restrict__ v) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ng) return;
    const double vm = v[gcells[gptr[g]]];
    for (int t = gptr[g] + 1; t < gptr[g + 1]; ++t) v[gcells[t]] = vm;
}

__global__ void k_group_fold(int ng, const int* __restrict__ gptr, const int* __restrict__ gcells,
                             double* __restrict__ v, int zero_slaves) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ng) return;
    double s = 0.0;
    for (int t = gptr[g]; t < gptr[g + 1]; ++t) s += v[gcells[t]];
    v[gcells[gptr[g]]] = s;
    for (int t = gptr[g] + 1; t < gptr[g + 1]; ++t) v[gcells[t]] = zero_slaves ? 0.0 : s;
}

int grid_for(long long n) {
    long long b = (n + kNT - 1) / kNT;
    long long cap = (long long)num_sms() * 16;
    return int(std::max(1LL, std::min(b, cap)));
}

}  // namespace

void launch_group_expand(vofp_ctx* c, double* v) {
    if (c->ngroups == 0) return;
    launch(c, k_group_expand, ceil_div(c->ngroups, kNT), kNT, c->stream, c->ngroups, c->gptr, c->gcells, v);
}

void launch_group_fold(vofp_ctx* c, double* v, bool zero_slaves) {
    if (c->ngroups == 0) return;
    launch(c, k_group_fold, ceil_div(c->ngroups, kNT), kNT, c->stream, c->ngroups, c->gptr, c->gcells, v,
                                                                    zero_slaves ? 1 : 0);
}

// Resolve merge chains on the host: the root of a small cell is the end of its target chain;
// a cycle of small cells is rooted at its member of largest open volume (lowest index on ties).
// Small cells are addressed by their slot in the lists (any order): tslot[t] is the slot of the
// target of slot t, -1 when the target does not merge. The roots do not depend on the order.
static void resolve_roots(const std::vector<long long>& cells, const std::vector<long long>& targets,
                          const std::vector<double>& vfs, const std::vector<int32_t>& tslot,
                          std::vector<long long>& roots) {
    const long long m = (long long)cells.size();
    std::vector<long long> root(m, -1);      // resolved root cell per slot
    std::vector<long long> stamp(m, -1);     // first slot of the walk that last visited it
    std::vector<long long> where(m, 0);      // its index on that walk's path
    std::vector<long long> path;
    for (long long t0 = 0; t0 < m; ++t0) {
        if (root[t0] >= 0) continue;
        path.clear();
        long long q = t0, r;
        while (true) {
            if (root[q] >= 0) {
                r = root[q];
                break;
            }
            if (stamp[q] == t0) {
                // a cycle: path[where[q]] .. the end
                long long best = -1;
                double bv = -1.0;
                for (size_t k = (size_t)where[q]; k < path.size(); ++k) {
                    const long long cm = cells[path[k]];
                    const double vm = vfs[path[k]];
                    if (vm > bv || (vm == bv && cm < best)) {
                        bv = vm;
                        best = cm;
                    }
                }
                for (size_t k = (size_t)where[q]; k < path.size(); ++k) root[path[k]] = best;
                r = best;
                break;
            }
            stamp[q] = t0;
            where[q] = (long long)path.size();
            path.push_back(q);
            if (tslot[q] < 0) {
                r = targets[q];   // the chain ends at a cell that does not merge
                break;
            }
            q = tslot[q];
        }
        for (long long k : path)
            if (root[k] < 0) root[k] = r;
    }
    roots.assign(root.begin(), root.end());
}

// Device lists of the small cells, kept across operator builds and grown when they overflow.
static vofp_status grow_small(vofp_ctx* c, long long cap) {
    void* old[4] = {c->small_cells, c->small_targets, c->small_vf, c->small_tslot};
    for (void* p : old)
        if (p) {
            cudaFree(p);
            c->allocs.erase(std::remove(c->allocs.begin(), c->allocs.end(), p), c->allocs.end());
        }
    c->bytes -= c->small_cap * (long long)(2 * sizeof(long long) + sizeof(double) + sizeof(int32_t));
    c->small_cells = c->small_targets = nullptr;
    c->small_vf = nullptr;
    c->small_tslot = nullptr;
    c->small_cap = 0;
    vofp_status s;
    if ((s = c->alloc(&c->small_cells, cap)) || (s = c->alloc(&c->small_targets, cap)) ||
        (s = c->alloc(&c->small_vf, cap)) || (s = c->alloc(&c->small_tslot, cap)))
        return s;
    c->small_cap = cap;
    return VOFP_OK;
}

// Group arrays (offsets, cells, corrections), kept across builds and grown when too small.
static vofp_status grow_groups(vofp_ctx* c, long long ng, long long ncells) {
    if (ng + 1 <= c->gptr_cap && ncells <= c->gcells_cap) return VOFP_OK;
    void* old[3] = {c->gptr, c->gcells, c->gcorr};
    for (void* p : old)
        if (p) {
            cudaFree(p);
            c->allocs.erase(std::remove(c->allocs.begin(), c->allocs.end(), p), c->allocs.end());
        }
    c->bytes -= c->gptr_cap * (long long)(sizeof(int) + sizeof(double)) + c->gcells_cap * (long long)sizeof(int);
    c->gptr = c->gcells = nullptr;
    c->gcorr = nullptr;
    c->gptr_cap = c->gcells_cap = 0;
    const long long pc = (ng + 1) * 3 / 2 + 16, cc = ncells * 3 / 2 + 16;
    vofp_status s;
    if ((s = c->alloc(&c->gptr, pc)) || (s = c->alloc(&c->gcells, cc)) || (s = c->alloc(&c->gcorr, pc))) return s;
    c->gptr_cap = pc;
    c->gcells_cap = cc;
    return VOFP_OK;
}

vofp_status build_operator(vofp_ctx* c, const double* F, const double* ax, const double* ay,
                           const double* az, const double* vf, const vofp_bc* bc,
                           const vofp_phys* phys) {
    const Dims d = c->d;
    const long long N = d.n;
    const long long nfx = (long long)(d.nx + 1) * d.ny * d.nz;
    const long long nfy = (long long)d.nx * (d.ny + 1) * d.nz;
    const long long nfz = (long long)d.nx * d.ny * (d.nz + 1);
    cudaStream_t st = c->stream;
    vofp_status s;
    if (!c->Tx) {
        if ((s = c->alloc(&c->Tx, N)) || (s = c->alloc(&c->Ty, N)) || (s = c->alloc(&c->Tz, N)) ||
            (s = c->alloc(&c->diag, N)) || (s = c->alloc(&c->axe, nfx)) || (s = c->alloc(&c->aye, nfy)) ||
            (s = c->alloc(&c->aze, nfz)) || (s = c->alloc(&c->s, N)) || (s = c->alloc(&c->sq, N)) ||
            (s = c->alloc(&c->Txs, N)) || (s = c->alloc(&c->Tys, N)) || (s = c->alloc(&c->Tzs, N)) ||
            (s = c->alloc(&c->Txf, N)) || (s = c->alloc(&c->Tyf, N)) || (s = c->alloc(&c->Tzf, N)) ||
            (s = c->alloc(&c->Tzr, N)) || (s = c->alloc(&c->rho, N)) || (s = c->alloc(&c->kx, N)) ||
            (s = c->alloc(&c->ky, N)) || (s = c->alloc(&c->kz, N)) ||
            (s = c->alloc(&c->slave_bits, (N + 31) / 32)) || (s = c->alloc(&c->root, N)) ||
            (s = c->alloc(&c->red_bits, (N + 31) / 32)) || (s = c->alloc(&c->excl_bits, (N + 31) / 32)) ||
            (s = c->alloc(&c->inactive, N)) || (s = c->alloc(&c->work, N)) ||
            (s = c->alloc(&c->partials, kMaxPartials)) || (s = c->alloc(&c->counters, 64)) ||
            (s = c->alloc(&c->sc, 4)))
            return s;
        VOFP_CUDA_TRY(c, cudaMemsetAsync(c->counters, 0, 64 * sizeof(unsigned int), st));
    }
    c->built = false;
    c->rbc_built = false;
    c->rbc_ok = false;
    for (int f = 0; f < 6; ++f) c->bc[f] = bc->kind[f];
    c->phys = *phys;
    c->dirichlet = false;
    Bc6 b6;
    for (int f = 0; f < 6; ++f) {
        b6.k[f] = bc->kind[f];
        c->dirichlet |= bc->kind[f] == VOFP_BC_DIRICHLET;
    }
    const int gN = grid_for(N);

    // density (Eq. density), optional smoothing (Sec. 2.10); rho lives in Txs during assembly
    double* rho = c->Txs;
    double* tmp = c->Tys;
    launch(c, k_density, gN, kNT, st, d, F, phys->rho_liquid, phys->rho_gas, rho);
    if (phys->density_smoothing) {
        for (int axis = 0; axis < 3; ++axis) {
            launch(c, k_smooth, gN, kNT, st, d, axis, rho, tmp);
            std::swap(rho, tmp);
        }
    }
    VOFP_CUDA_TRY(c, cudaMemcpyAsync(c->rho, rho, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
    // activity, iterated to a fixed point
    uint8_t* ina_a = c->inactive;
    uint8_t* ina_b = reinterpret_cast<uint8_t*>(c->work);
    launch(c, k_activity_init, gN, kNT, st, d, vf, ina_a);
    unsigned int* changed = c->counters + 32;
    for (int pass = 0; pass < 100000; ++pass) {
        VOFP_CUDA_TRY(c, cudaMemsetAsync(changed, 0, sizeof(unsigned int), st));
        launch(c, k_activity_step, gN, kNT, st, d, b6, ax, ay, az, ina_a, ina_b, changed);
        unsigned int h = 0;
        VOFP_CUDA_TRY(c, cudaMemcpyAsync(&h, changed, sizeof(h), cudaMemcpyDeviceToHost, st));
        VOFP_CUDA_TRY(c, cudaStreamSynchronize(st));
        std::swap(ina_a, ina_b);
        if (h == 0) break;
    }
    if (ina_a != c->inactive)
        VOFP_CUDA_TRY(c, cudaMemcpyAsync(c->inactive, ina_a, N, cudaMemcpyDeviceToDevice, st));
    {
        unsigned int* ninact = c->counters + 34;
        VOFP_CUDA_TRY(c, cudaMemsetAsync(ninact, 0, sizeof(unsigned int), st));
        launch(c, k_count_u8, gN, kNT, st, d.n, c->inactive, ninact);
        unsigned int h = 0;
        VOFP_CUDA_TRY(c, cudaMemcpyAsync(&h, ninact, sizeof(h), cudaMemcpyDeviceToHost, st));
        VOFP_CUDA_TRY(c, cudaStreamSynchronize(st));
        c->n_inactive = h;
    }
    // prescribed Neumann fluxes are copied so the caller's arrays need not outlive this call
    for (int f = 0; f < 6; ++f) {
        const long long nb = f < 2 ? (long long)d.ny * d.nz : f < 4 ? (long long)d.nx * d.nz : (long long)d.nx * d.ny;
        if (bc->neumann_flux[f] && bc->kind[f] == VOFP_BC_NEUMANN) {
            if (!c->nflux[f] && (s = c->alloc(&c->nflux[f], nb))) return s;
            VOFP_CUDA_TRY(c, cudaMemcpyAsync(c->nflux[f], bc->neumann_flux[f], sizeof(double) * nb,
                                             cudaMemcpyDeviceToDevice, st));
            c->has_nflux[f] = true;
        } else {
            c->has_nflux[f] = false;
        }
    }
    launch(c, k_eff_apertures, grid_for(nfx + nfy + nfz), kNT, st, d, ax, ay, az, c->inactive, c->axe, c->aye, c->aze);
    if (d.nx % 2 == 0) {
        // x-pairs of cells, 16-byte words on the cell and y/z-face streams
        const int gP = grid_for(d.n / 2);
        launch(c, k_face_coeffs2, gP, kNT, st, d, c->dx, c->dy, c->dz, rho, c->axe, c->aye, c->aze, c->Tx, c->Ty,
               c->Tz, c->kx, c->ky, c->kz);
        launch(c, k_diag2, gP, kNT, st, d, b6, c->dx, c->dy, c->dz, rho, c->axe, c->aye, c->aze, c->Tx, c->Ty, c->Tz,
               c->diag);
    } else {
        launch(c, k_face_coeffs, gN, kNT, st, d, c->dx, c->dy, c->dz, rho, c->axe, c->aye, c->aze, c->Tx, c->Ty,
               c->Tz, c->kx, c->ky, c->kz);
        launch(c, k_diag, gN, kNT, st, d, b6, c->dx, c->dy, c->dz, rho, c->axe, c->aye, c->aze, c->Tx, c->Ty, c->Tz,
               c->diag);
    }

    // merge map (Sec. 2.3): small cells listed on the device, chains resolved on the host
    std::vector<long long> cells, targets, roots;
    std::vector<double> vfs;
    std::vector<int32_t> tslot;
    unsigned int* cnt = c->counters + 33;
    if (vf && phys->merge_threshold > 0.0) {
        unsigned int m = 0;
        for (int attempt = 0; attempt < 2; ++attempt) {
            VOFP_CUDA_TRY(c, cudaMemsetAsync(cnt, 0, sizeof(unsigned int), st));
            launch(c, k_small_cells, gN, kNT, st, d, phys->merge_threshold, vf, c->inactive, c->dx, c->dy, c->dz,
                   c->axe, c->aye, c->aze, cnt, c->small_cap, c->small_cells, c->small_targets, c->small_vf);
            VOFP_CUDA_TRY(c, cudaMemcpyAsync(&m, cnt, sizeof(m), cudaMemcpyDeviceToHost, st));
            VOFP_CUDA_TRY(c, cudaStreamSynchronize(st));
            if ((long long)m <= c->small_cap) break;
            if ((s = grow_small(c, (long long)m + m / 2 + 1024))) return s;
        }
        if ((long long)m > c->small_cap) {
            c->set_error("small-cell count changed between two passes over the same input");
            return VOFP_ERR_CUDA;
        }
        if (m > 0) {
            // root[] serves as the cell -> slot map here; k_root_init below rewrites it
            VOFP_CUDA_TRY(c, cudaMemsetAsync(c->root, 0xff, sizeof(int32_t) * N, st));
            launch(c, k_small_slots, ceil_div(m, kNT), kNT, st, (int)m, (const long long*)c->small_cells, c->root);
            launch(c, k_small_target_slots, ceil_div(m, kNT), kNT, st, (int)m, (const long long*)c->small_targets,
                   (const int32_t*)c->root, c->small_tslot);
            cells.resize(m);
            targets.resize(m);
            vfs.resize(m);
            tslot.resize(m);
            VOFP_CUDA_TRY(c, cudaMemcpyAsync(cells.data(), c->small_cells, sizeof(long long) * m,
                                             cudaMemcpyDeviceToHost, st));
            VOFP_CUDA_TRY(c, cudaMemcpyAsync(targets.data(), c->small_targets, sizeof(long long) * m,
                                             cudaMemcpyDeviceToHost, st));
            VOFP_CUDA_TRY(c, cudaMemcpyAsync(vfs.data(), c->small_vf, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
            VOFP_CUDA_TRY(c, cudaMemcpyAsync(tslot.data(), c->small_tslot, sizeof(int32_t) * m,
                                             cudaMemcpyDeviceToHost, st));
            VOFP_CUDA_TRY(c, cudaStreamSynchronize(st));
        }
    }
    resolve_roots(cells, targets, vfs, tslot, roots);
    launch(c, k_root_init, gN, kNT, st, d, c->inactive, c->root);
    // groups: cells whose root differs from themselves, plus the roots
    std::vector<std::pair<long long, long long>> members;   // (root, cell)
    for (size_t t = 0; t < cells.size(); ++t)
        if (roots[t] != cells[t]) members.push_back({roots[t], cells[t]});
    std::sort(members.begin(), members.end());
    std::vector<int> gptr(1, 0), gcells;
    for (size_t t = 0; t < members.size();) {
        long long r = members[t].first;
        gcells.push_back((int)r);
        while (t < members.size() && members[t].first == r) gcells.push_back((int)members[t++].second);
        gptr.push_back((int)gcells.size());
    }
    c->ngroups = (int)gptr.size() - 1;
    c->n_merged = (long long)members.size();
    c->n_unknowns = N - c->n_inactive - c->n_merged;
    if (c->ngroups > 0) {
        if ((s = grow_groups(c, c->ngroups, (long long)gcells.size()))) return s;
        VOFP_CUDA_TRY(c, cudaMemcpyAsync(c->gptr, gptr.data(), sizeof(int) * gptr.size(), cudaMemcpyHostToDevice, st));
        VOFP_CUDA_TRY(c, cudaMemcpyAsync(c->gcells, gcells.data(), sizeof(int) * gcells.size(), cudaMemcpyHostToDevice, st));
        // (cell, root) of every merged cell, through the small-cell lists (there are no more
        // merged cells than small cells); copies from pageable host memory are staged before
        // cudaMemcpyAsync returns, so the vectors may go out of scope
        std::vector<long long> mc, mr;
        mc.reserve(members.size());
        mr.reserve(members.size());
        for (auto& pr : members) {
            mc.push_back(pr.second);
            mr.push_back(pr.first);
        }
        VOFP_CUDA_TRY(c, cudaMemcpyAsync(c->small_cells, mc.data(), sizeof(long long) * mc.size(),
                                         cudaMemcpyHostToDevice, st));
        VOFP_CUDA_TRY(c, cudaMemcpyAsync(c->small_targets, mr.data(), sizeof(long long) * mr.size(),
                                         cudaMemcpyHostToDevice, st));
        launch(c, k_root_scatter, ceil_div((long long)mc.size(), kNT), kNT, st, (int)mc.size(),
               (const long long*)c->small_cells, (const long long*)c->small_targets, c->root);
    }
    // symmetric scaling s = diag(A_hat)^-1/2 per group
    launch(c, k_scale_cells, gN, kNT, st, d, c->inactive, c->diag, c->s, c->sq);
    if (c->ngroups > 0)
        launch(c, k_scale_groups, ceil_div(c->ngroups, kNT), kNT, st, d, c->ngroups, c->gptr, c->gcells, c->root, c->diag,
                                                                  c->Tx, c->Ty, c->Tz, c->s, c->sq, c->gcorr);
    launch(c, k_scaled_coeffs, gN, kNT, st, d, c->s, c->Tx, c->Ty, c->Tz, c->Txs, c->Tys, c->Tzs, c->Txf, c->Tyf, c->Tzf);
    launch(c, k_slave_bits, grid_for((N + 31) / 32), kNT, st, d, c->root, c->slave_bits);
    {
        unsigned int* nred = c->counters + 35;
        VOFP_CUDA_TRY(c, cudaMemsetAsync(nred, 0, sizeof(unsigned int), st));
        launch(c, k_red_bits, grid_for((N + 31) / 32), kNT, st, d, (const int32_t*)c->root,
               (const uint32_t*)c->slave_bits, c->red_bits, c->excl_bits, nred);
        launch(c, k_signed_tz, gN, kNT, st, d.n, (const float*)c->Tzf, (const uint32_t*)c->red_bits, c->Tzr);
        unsigned int h = 0;
        VOFP_CUDA_TRY(c, cudaMemcpyAsync(&h, nred, sizeof(h), cudaMemcpyDeviceToHost, st));
        VOFP_CUDA_TRY(c, cudaStreamSynchronize(st));
        c->n_red = h;
    }
    VOFP_CUDA_TRY(c, cudaGetLastError());
    VOFP_CUDA_TRY(c, cudaStreamSynchronize(st));
    c->built = true;
    return VOFP_OK;
}

vofp_status rhs(vofp_ctx* c, const double* u, const double* v, const double* w, const double* body,
                double* b) {
    const Dims d = c->d;
    Bc6 b6;
    for (int f = 0; f < 6; ++f) b6.k[f] = c->bc[f];
    Flux6 nf{};
    for (int f = 0; f < 6; ++f) nf.g[f] = c->has_nflux[f] ? c->nflux[f] : nullptr;
    launch(c, k_rhs, grid_for(d.n), kNT, c->stream, d, b6, nf, c->phys.dt, c->dx, c->dy, c->dz, c->axe, c->aye,
                                                c->aze, c->inactive, u, v, w, body, b);
    VOFP_CUDA_TRY(c, cudaGetLastError());
    return VOFP_OK;
}

}  // namespace vofp
