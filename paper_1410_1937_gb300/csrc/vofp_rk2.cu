// One second-order Runge-Kutta step of Sec. 2.1 around the pressure solve, composed of the
// library's own calls on the context stream:
//   stage 1  operator with rho(phi^k); solve for P* with the face field u^k + dt R (Eq. poisson1),
//            warm-started from the caller's pressure; u* = u^k + dt (R - grad P* / rho) (Eq. runge1);
//            phi* = phi^k - VOF(u^k, phi^k, dt);
//   stage 2  operator with rho(phi*); solve for P^{k+1} with the face field u* + u^k + dt R
//            (Eq. poisson2), warm-started from P*; u^{k+1} = (u* + u^k + dt (R - grad P^{k+1} / rho)) / 2
//            (Eq. runge2); phi^{k+1} = phi^k - VOF((u* + u^k) / 2, phi^k, dt).
// The face field handed to the right-hand side and the projection is the velocity the paper's
// divergence acts on: b = -(1/dt) div(field) and field - dt grad P / rho.
#include <algorithm>

#include "vofp_internal.cuh"

namespace vofp {
namespace {

constexpr int kNT = 256;

// out = a x + b y + c z (y, z may be null)
__global__ void k_axpbypcz(long long n, double a, const double* __restrict__ x, double b, const double* __restrict__ y,
                           double c, const double* __restrict__ z, double* __restrict__ out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double v = a * x[i];
        if (y) v = fma(b, y[i], v);
        if (z) v = fma(c, z[i], v);
        out[i] = v;
    }
}

void combine(vofp_ctx* c, long long n, double a, const double* x, double b, const double* y, double cc,
             const double* z, double* out) {
    const int g = (int)std::max(1LL, std::min((n + kNT - 1) / kNT, (long long)num_sms() * 8));
    launch(c, k_axpbypcz, g, kNT, c->stream, n, a, x, b, y, cc, z, out);
}

}  // namespace
}  // namespace vofp

extern "C" vofp_status vofp_rk2_step(vofp_ctx* c, double* F, const double* ax, const double* ay, const double* az,
                                     const double* vf, double* u, double* v, double* w, const double* Ru,
                                     const double* Rv, const double* Rw, const vofp_bc* bc, const vofp_phys* phys,
                                     const vofp_solve_opts* opts, double* p, int order, vofp_rk2_info* info) {
    using namespace vofp;
    if (!c) return VOFP_ERR_INVALID_ARG;
    if (!F || !ax || !ay || !az || !vf || !u || !v || !w || !bc || !phys || !opts || !p) {
        c->set_error("null input");
        return VOFP_ERR_INVALID_ARG;
    }
    if ((Ru != nullptr) != (Rv != nullptr) || (Ru != nullptr) != (Rw != nullptr)) {
        c->set_error("R must be given for all three face arrays or for none");
        return VOFP_ERR_INVALID_ARG;
    }
    const Dims d = c->d;
    const long long N = d.n, nfx = (long long)(d.nx + 1) * d.ny * d.nz, nfy = (long long)d.nx * (d.ny + 1) * d.nz,
                    nfz = (long long)d.nx * d.ny * (d.nz + 1);
    const long long nf[3] = {nfx, nfy, nfz};
    vofp_status s;
    if (!c->rk2_buf) {
        // three face fields (field, u*, midpoint velocity) and three cell arrays (phi*, b, P*)
        if ((s = c->alloc(&c->rk2_buf, 3 * (nfx + nfy + nfz) + 3 * N))) return s;
    }
    double* fld[3] = {c->rk2_buf, c->rk2_buf + nfx, c->rk2_buf + nfx + nfy};
    double* ust[3] = {fld[2] + nfz, fld[2] + nfz + nfx, fld[2] + nfz + nfx + nfy};
    double* mid[3] = {ust[2] + nfz, ust[2] + nfz + nfx, ust[2] + nfz + nfx + nfy};
    double* phis = mid[2] + nfz;
    double* b = phis + N;
    double* pst = b + N;
    double* vel[3] = {u, v, w};
    const double* R[3] = {Ru, Rv, Rw};
    const double dt = phys->dt;
    vofp_solve_opts o = *opts;
    o.x0_zero = 0;
    vofp_rk2_info local{};
    vofp_rk2_info* inf = info ? info : &local;

    // stage 1
    if ((s = vofp_build_operator(c, F, ax, ay, az, vf, bc, phys))) return s;
    for (int a = 0; a < 3; ++a) combine(c, nf[a], 1.0, vel[a], dt, R[a], 0.0, nullptr, fld[a]);
    if ((s = vofp_rhs_from_face_velocity(c, fld[0], fld[1], fld[2], nullptr, b))) return s;
    VOFP_CUDA_TRY(c, cudaMemcpyAsync(pst, p, sizeof(double) * N, cudaMemcpyDeviceToDevice, c->stream));
    s = vofp_solve(c, b, pst, &o, &inf->solve1);
    if (s) return s;
    if ((s = vofp_project(c, pst, fld[0], fld[1], fld[2], nullptr, ust[0], ust[1], ust[2], nullptr, nullptr))) return s;
    if ((s = vofp_vof_advect(c, F, ax, ay, az, vf, u, v, w, dt, order, phis))) return s;

    // stage 2
    if ((s = vofp_build_operator(c, phis, ax, ay, az, vf, bc, phys))) return s;
    for (int a = 0; a < 3; ++a) {
        combine(c, nf[a], 1.0, ust[a], 1.0, vel[a], dt, R[a], fld[a]);
        combine(c, nf[a], 0.5, ust[a], 0.5, vel[a], 0.0, nullptr, mid[a]);
    }
    if ((s = vofp_rhs_from_face_velocity(c, fld[0], fld[1], fld[2], nullptr, b))) return s;
    VOFP_CUDA_TRY(c, cudaMemcpyAsync(p, pst, sizeof(double) * N, cudaMemcpyDeviceToDevice, c->stream));
    s = vofp_solve(c, b, p, &o, &inf->solve2);
    if (s) return s;
    // u^{k+1} = (field - dt grad P^{k+1} / rho) / 2, written over u, v, w
    if ((s = vofp_project(c, p, fld[0], fld[1], fld[2], nullptr, fld[0], fld[1], fld[2], nullptr, &inf->max_div)))
        return s;
    for (int a = 0; a < 3; ++a) combine(c, nf[a], 0.5, fld[a], 0.0, nullptr, 0.0, nullptr, vel[a]);
    inf->max_div *= 0.5;
    if ((s = vofp_vof_advect(c, F, ax, ay, az, vf, mid[0], mid[1], mid[2], dt, order, F))) return s;
    VOFP_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return VOFP_OK;
}
