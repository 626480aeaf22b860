// VOF operator of Sec. 2.4: flux-error correction and operator-split advection of the volume
// fraction with a dilation term (FP64).
//
// Correction (one pass over the cells): face fluxes F = A (u - v) with A the open face area
// (aperture x face area) and u - v the relative velocity given on the faces; the cell's
// conservation error E = sum_i (F+_i - F-_i) (Eq. diverge) is removed along z,
//   F~+_z = F+_z - E A+_z / (A+_z + A-_z),   F~-_z = F-_z + E A-_z / (A+_z + A-_z),
// and the stage velocities are u^_i = dx_i F~_i / V = F~_i / (uncut face area): shared on x and y
// faces, per cell on z faces (the two cells of a z face may disagree).
//
// Stage along axis d (two passes): the piecewise-linear interface of every cell with 0 < phi < 1
// (normal m = -grad phi by central differences weighted (1, 2, 1) x (1, 2, 1) across the other
// axes; plane constant alpha with the fluid volume {m.x <= alpha} equal to phi V, by Newton steps),
// then per cell the fluid carried through its two d faces in slabs of thickness |u^| dt of the
// donor cell (the cell itself on outflow, the neighbour on inflow; the boundary cell on inflow
// through a domain face), and
//   implicit stage:  phi_new = (phi - (F+ - F-) / V) / (1 - dt (u^+ - u^-) / dx_d)
//   explicit stage:  phi_new =  phi - (F+ - F-) / V + dt phi (u^+ - u^-) / dx_d.
// The first two stages are implicit, the third explicit; the axes run x, y, z (order 0) or
// z, y, x (order 1).  Neighbours inside the body (no open volume) and outside the domain take the
// cell's own value in the normal; a slab is at most the donor cell; phi is not clipped.
#include <algorithm>

#include "vofp_internal.cuh"

namespace vofp {
namespace {

constexpr int kNT = 256;

int grid_cells(long long n) {
    return (int)std::max(1LL, std::min((n + kNT - 1) / kNT, (long long)num_sms() * 16));
}

// ---- fluid volume below a plane in a box -------------------------------------------------------

// volume fraction of {y in [0,1]^3 : c.y <= b} for sorted c1 <= c2 <= c3, sum 1, b in [0, 1]
__device__ double cube_fraction(double c1, double c2, double c3, double b) {
    const bool flip = b > 0.5;
    if (flip) b = 1.0 - b;
    double f;
    if (b <= 0.0) {
        f = 0.0;
    } else {
        const double c12 = c1 + c2;
        if (b < c1) {
            f = b * (b / c1) * b / (6.0 * c2 * c3);
        } else if (b < c2) {
            f = (b * (b - c1) + c1 * c1 / 3.0) / (2.0 * c2 * c3);
        } else {
            const double p1 = 3.0 * b * b - 3.0 * b * c1 + c1 * c1;
            const double e2 = b - c2;
            if (b < fmin(c12, c3)) {
                f = (p1 - e2 * (e2 / c1) * e2) / (6.0 * c2 * c3);
            } else if (c3 < c12) {
                const double e3 = b - c3;
                f = (p1 - e2 * (e2 / c1) * e2 - e3 * (e3 / c1) * e3) / (6.0 * c2 * c3);
            } else {
                f = (2.0 * b - c12) / (2.0 * c3);
            }
        }
    }
    return flip ? 1.0 - f : f;
}

__device__ __forceinline__ void sort3(double& a, double& b, double& c) {
    if (a > b) { const double t = a; a = b; b = t; }
    if (b > c) { const double t = b; b = c; c = t; }
    if (a > b) { const double t = a; a = b; b = t; }
}

// the unit-cube fraction of one cell's normal with its divisions done once (for the bisection)
struct CubeFrac {
    double c1, c2, c3, ic1, k6, k2, k5;
    __device__ CubeFrac(double a1, double a2, double a3) {
        sort3(a1, a2, a3);
        c1 = a1;
        c2 = a2;
        c3 = a3;
        ic1 = c1 > 0.0 ? 1.0 / c1 : 0.0;
        k6 = 1.0 / (6.0 * c2 * c3);
        k2 = 1.0 / (2.0 * c2 * c3);
        k5 = 1.0 / (2.0 * c3);
    }
    __device__ double operator()(double b) const {
        const bool flip = b > 0.5;
        if (flip) b = 1.0 - b;
        double f;
        if (b <= 0.0) {
            f = 0.0;
        } else {
            const double c12 = c1 + c2;
            if (b < c1) {
                f = b * (b * ic1) * b * k6;
            } else if (b < c2) {
                f = (b * (b - c1) + c1 * c1 / 3.0) * k2;
            } else {
                const double p1 = 3.0 * b * b - 3.0 * b * c1 + c1 * c1;
                const double e2 = b - c2;
                if (b < fmin(c12, c3)) {
                    f = (p1 - e2 * (e2 * ic1) * e2) * k6;
                } else if (c3 < c12) {
                    const double e3 = b - c3;
                    f = (p1 - e2 * (e2 * ic1) * e2 - e3 * (e3 * ic1) * e3) * k6;
                } else {
                    f = (2.0 * b - c12) * k5;
                }
            }
        }
        return flip ? 1.0 - f : f;
    }
    // d/db of the fraction: the area of the cut, region by region (the fraction is symmetric,
    // f(b) = 1 - f(1 - b), so its derivative at b is the one at 1 - b)
    __device__ double deriv(double b) const {
        if (b > 0.5) b = 1.0 - b;
        if (b <= 0.0) return 0.0;
        const double c12 = c1 + c2;
        if (b < c1) return b * (b * ic1) * (3.0 * k6);
        if (b < c2) return (2.0 * b - c1) * k2;
        const double e2 = b - c2;
        if (b < fmin(c12, c3)) return (2.0 * b - c1 - e2 * (e2 * ic1)) * k2;
        if (c3 < c12) {
            const double e3 = b - c3;
            return (2.0 * b - c1 - e2 * (e2 * ic1) - e3 * (e3 * ic1)) * k2;
        }
        return 2.0 * k5;
    }
};

// volume of {x in [0,h] : m.x <= alpha}
__device__ double box_volume(double mx, double my, double mz, double alpha, double hx, double hy, double hz) {
    // reflect negative components (x -> h - x)
    if (mx < 0) alpha -= mx * hx;
    if (my < 0) alpha -= my * hy;
    if (mz < 0) alpha -= mz * hz;
    double a1 = fabs(mx) * hx, a2 = fabs(my) * hy, a3 = fabs(mz) * hz;
    const double s = (a1 + a2) + a3;
    const double vol = (hx * hy) * hz;
    if (alpha <= 0.0) return 0.0;
    if (alpha >= s) return vol;
    const double is = 1.0 / s;
    a1 *= is;
    a2 *= is;
    a3 *= is;
    sort3(a1, a2, a3);
    return cube_fraction(a1, a2, a3, alpha * is) * vol;
}

// ---- correction --------------------------------------------------------------------------------

__global__ void k_vof_correct(Dims d, const double* __restrict__ dx, const double* __restrict__ dy,
                              const double* __restrict__ dz, const double* __restrict__ ax,
                              const double* __restrict__ ay, const double* __restrict__ az,
                              const double* __restrict__ u, const double* __restrict__ v,
                              const double* __restrict__ w, double* __restrict__ uxh, double* __restrict__ uyh,
                              double* __restrict__ wmh, double* __restrict__ wph) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < d.n; c += (long long)gridDim.x * blockDim.x) {
        int i, j, k;
        cell_ijk(d, c, i, j, k);
        const double Sx = dz[k] * dy[j], Sy = dz[k] * dx[i], Sz = dy[j] * dx[i];
        const long long fxm = fx_idx(d, i, j, k), fym = fy_idx(d, i, j, k), fzm = fz_idx(d, i, j, k);
        const long long fxp = fxm + 1, fyp = fym + d.nx, fzp = fzm + d.plane;
        const double Fxm = (ax[fxm] * Sx) * u[fxm], Fxp = (ax[fxp] * Sx) * u[fxp];
        const double Fym = (ay[fym] * Sy) * v[fym], Fyp = (ay[fyp] * Sy) * v[fyp];
        const double Am = az[fzm] * Sz, Ap = az[fzp] * Sz;
        const double Fzm = Am * w[fzm], Fzp = Ap * w[fzp];
        const double E = ((Fxp - Fxm) + (Fyp - Fym)) + (Fzp - Fzm);
        const double tot = Ap + Am;
        const double share = tot > 0.0 ? E / tot : 0.0;
        const double iSz = 1.0 / Sz;
        wph[c] = (Fzp - share * Ap) * iSz;
        wmh[c] = (Fzm + share * Am) * iSz;
        // u^ = F / S = aperture x velocity on the x and y faces
        uxh[fxm] = ax[fxm] * u[fxm];
        if (i == d.nx - 1) uxh[fxp] = ax[fxp] * u[fxp];
        uyh[fym] = ay[fym] * v[fym];
        if (j == d.ny - 1) uyh[fyp] = ay[fyp] * v[fyp];
    }
}

// ---- reconstruction ----------------------------------------------------------------------------

__device__ __forceinline__ double span(const double* __restrict__ w, int i, int n) {
    const double wp = i > 0 ? w[i - 1] : w[i], wn = i < n - 1 ? w[i + 1] : w[i];
    return 0.5 * wp + w[i] + 0.5 * wn;
}

// (m, alpha) of every cell with 0 < phi < 1 (m = 0 elsewhere)
__global__ void k_vof_plic(Dims d, const double* __restrict__ dx, const double* __restrict__ dy,
                           const double* __restrict__ dz, const double* __restrict__ vf,
                           const double* __restrict__ phi, double4* __restrict__ plic) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < d.n; c += (long long)gridDim.x * blockDim.x) {
        const double pc = phi[c];
        if (!(pc > 0.0 && pc < 1.0)) {
            plic[c] = make_double4(0.0, 0.0, 0.0, 0.0);
            continue;
        }
        int i, j, k;
        cell_ijk(d, c, i, j, k);
        double val[3][3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                for (int e = 0; e < 3; ++e) {
                    const int kk = k + a - 1, jj = j + b - 1, ii = i + e - 1;
                    double s = pc;
                    if (kk >= 0 && kk < d.nz && jj >= 0 && jj < d.ny && ii >= 0 && ii < d.nx) {
                        const long long q = ii + (long long)d.nx * (jj + (long long)d.ny * kk);
                        if (vf[q] > 0.0) s = phi[q];
                    }
                    val[a][b][e] = s;
                }
        const double wt[3] = {1.0, 2.0, 1.0};
        double gx = 0.0, gy = 0.0, gz = 0.0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                gx += wt[a] * wt[b] * (val[a][b][2] - val[a][b][0]);
                gy += wt[a] * wt[b] * (val[a][2][b] - val[a][0][b]);
                gz += wt[a] * wt[b] * (val[2][a][b] - val[0][a][b]);
            }
        const double mx = -(gx / 16.0) / span(dx, i, d.nx), my = -(gy / 16.0) / span(dy, j, d.ny),
                     mz = -(gz / 16.0) / span(dz, k, d.nz);
        const double hx = dx[i], hy = dy[j], hz = dz[k];
        // with x_i -> h_i - x_i for negative components the fluid is {a.y <= beta} in the unit
        // cube, a_i = |m_i| h_i / s, beta = (alpha - lo) / s, s = sum |m_i| h_i: Newton steps on
        // beta with the cut area as derivative, kept inside a bracket that bisects when a step
        // leaves it
        const double lo0 = fmin(mx * hx, 0.0) + fmin(my * hy, 0.0) + fmin(mz * hz, 0.0);
        const double a1 = fabs(mx) * hx, a2 = fabs(my) * hy, a3 = fabs(mz) * hz;
        const double sum = (a1 + a2) + a3;
        double alpha = 0.0;
        if (sum > 0.0) {
            const double is = 1.0 / sum;
            const CubeFrac f(a1 * is, a2 * is, a3 * is);
            double lo = 0.0, hi = 1.0, b = pc;
            for (int it = 0; it < 100; ++it) {
                const double r = f(b) - pc;
                if (r == 0.0) break;
                if (r < 0.0) lo = b;
                else hi = b;
                const double dv = f.deriv(b);
                double nb = dv > 0.0 ? b - r / dv : 0.5 * (lo + hi);
                if (!(nb > lo && nb < hi)) nb = 0.5 * (lo + hi);
                if (nb == b || fabs(nb - b) <= 2.3e-16 * b) {
                    b = nb;
                    break;
                }
                b = nb;
            }
            alpha = lo0 + b * sum;
        }
        plic[c] = make_double4(mx, my, mz, alpha);
    }
}

// ---- one stage ---------------------------------------------------------------------------------

// fluid in the slab of thickness t at the + or - face of a cell along `axis`
__device__ double slab(double ph, double4 pl, double hx, double hy, double hz, int axis, bool plus, double t) {
    double h[3] = {hx, hy, hz};
    const double m[3] = {pl.x, pl.y, pl.z};
    t = fmin(t, h[axis]);
    if (!(t > 0.0)) return 0.0;
    double alpha = pl.w;
    if (plus) alpha -= m[axis] * (h[axis] - t);
    h[axis] = t;
    const bool interface = ph > 0.0 && ph < 1.0 && (fabs(m[0]) + fabs(m[1]) + fabs(m[2])) > 0.0;
    if (!interface) return ph * ((h[0] * h[1]) * h[2]);
    return box_volume(m[0], m[1], m[2], alpha, h[0], h[1], h[2]);
}

__global__ void k_vof_stage(Dims d, int axis, int implicit, double dt, const double* __restrict__ dx,
                            const double* __restrict__ dy, const double* __restrict__ dz,
                            const double* __restrict__ phi, const double4* __restrict__ plic,
                            const double* __restrict__ uxh, const double* __restrict__ uyh,
                            const double* __restrict__ wmh, const double* __restrict__ wph,
                            double* __restrict__ out) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < d.n; c += (long long)gridDim.x * blockDim.x) {
        int i, j, k;
        cell_ijk(d, c, i, j, k);
        int idx[3] = {i, j, k};
        const int n[3] = {d.nx, d.ny, d.nz};
        const long long stride[3] = {1, (long long)d.nx, d.plane};
        double up, um;
        if (axis == 0) {
            const long long f = fx_idx(d, i, j, k);
            um = uxh[f];
            up = uxh[f + 1];
        } else if (axis == 1) {
            const long long f = fy_idx(d, i, j, k);
            um = uyh[f];
            up = uyh[f + d.nx];
        } else {
            um = wmh[c];
            up = wph[c];
        }
        const long long cn = idx[axis] < n[axis] - 1 ? c + stride[axis] : c;   // + neighbour (or self)
        const long long cp = idx[axis] > 0 ? c - stride[axis] : c;             // - neighbour (or self)
        auto width = [&](long long q, int which) -> double {
            // widths of cell q (same row/column as c except along `axis`)
            int ii = i, jj = j, kk = k;
            if (q != c) {
                if (axis == 0) ii += (q > c) ? 1 : -1;
                else if (axis == 1) jj += (q > c) ? 1 : -1;
                else kk += (q > c) ? 1 : -1;
            }
            return which == 0 ? dx[ii] : which == 1 ? dy[jj] : dz[kk];
        };
        const double pc = phi[c];
        const double4 lc = plic[c];
        const double hx = dx[i], hy = dy[j], hz = dz[k];
        double Fp, Fm;
        if (up > 0.0) {
            Fp = slab(pc, lc, hx, hy, hz, axis, true, up * dt);
        } else {
            Fp = -slab(phi[cn], plic[cn], width(cn, 0), width(cn, 1), width(cn, 2), axis, false, -up * dt);
        }
        if (um > 0.0) {
            Fm = slab(phi[cp], plic[cp], width(cp, 0), width(cp, 1), width(cp, 2), axis, true, um * dt);
        } else {
            Fm = -slab(pc, lc, hx, hy, hz, axis, false, -um * dt);
        }
        const double iV = 1.0 / ((hx * hy) * hz);
        const double other = axis == 0 ? hy * hz : axis == 1 ? hx * hz : hx * hy;   // V / dx_d
        const double adv = pc - (Fp - Fm) * iV;
        const double div = dt * (up - um) * (other * iV);
        out[c] = implicit ? adv / (1.0 - div) : adv + pc * div;
    }
}

}  // namespace

vofp_status vof_flux_correct(vofp_ctx* c, const double* ax, const double* ay, const double* az, const double* u,
                             const double* v, const double* w, double* uxh, double* uyh, double* wmh, double* wph) {
    launch(c, k_vof_correct, grid_cells(c->d.n), kNT, c->stream, c->d, (const double*)c->dx, (const double*)c->dy,
           (const double*)c->dz, ax, ay, az, u, v, w, uxh, uyh, wmh, wph);
    return VOFP_OK;
}

vofp_status vof_advect(vofp_ctx* c, const double* F, const double* ax, const double* ay, const double* az,
                       const double* vf, const double* u, const double* v, const double* w, double dt, int order,
                       double* F_out) {
    const Dims d = c->d;
    const long long N = d.n;
    vofp_status s;
    if (!c->vof_uxh) {
        if ((s = c->alloc(&c->vof_uxh, (long long)(d.nx + 1) * d.ny * d.nz)) ||
            (s = c->alloc(&c->vof_uyh, (long long)d.nx * (d.ny + 1) * d.nz)) || (s = c->alloc(&c->vof_wmh, N)) ||
            (s = c->alloc(&c->vof_wph, N)) || (s = c->alloc(&c->vof_phi, 2 * N)) ||
            (s = c->alloc(&c->vof_plic, 4 * N)))
            return s;
    }
    cudaStream_t st = c->stream;
    vof_flux_correct(c, ax, ay, az, u, v, w, c->vof_uxh, c->vof_uyh, c->vof_wmh, c->vof_wph);
    const int axes[2][3] = {{0, 1, 2}, {2, 1, 0}};
    const double* in = F;
    double4* plic = reinterpret_cast<double4*>(c->vof_plic);
    for (int stage = 0; stage < 3; ++stage) {
        double* out = stage == 2 ? F_out : c->vof_phi + (stage % 2) * N;
        launch(c, k_vof_plic, grid_cells(N), kNT, st, d, (const double*)c->dx, (const double*)c->dy,
               (const double*)c->dz, vf, in, plic);
        launch(c, k_vof_stage, grid_cells(N), kNT, st, d, axes[order ? 1 : 0][stage], stage < 2 ? 1 : 0, dt,
               (const double*)c->dx, (const double*)c->dy, (const double*)c->dz, in, (const double4*)plic,
               (const double*)c->vof_uxh, (const double*)c->vof_uyh, (const double*)c->vof_wmh,
               (const double*)c->vof_wph, out);
        in = out;
    }
    return VOFP_OK;
}

}  // namespace vofp
