// extern "C" entry points of libvofp (declared and documented in include/vofp.h): argument
// checks, context lifetime and error reporting around the implementations in the other files.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "vofp_internal.cuh"

namespace {

const char* kNullCtx = "null context";

vofp_status check_ctx(vofp_ctx* c, bool need_built) {
    if (!c) return VOFP_ERR_INVALID_ARG;
    c->err.clear();
    if (need_built && !c->built) {
        c->set_error("vofp_build_operator has not succeeded on this context");
        return VOFP_ERR_NOT_BUILT;
    }
    return VOFP_OK;
}

vofp_status invalid(vofp_ctx* c, const char* m) {
    if (c) c->set_error(m);
    return VOFP_ERR_INVALID_ARG;
}

vofp_status fail_cuda(vofp_ctx* c) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        c->set_error(std::string("kernel launch: ") + cudaGetErrorString(e));
        return VOFP_ERR_CUDA;
    }
    return VOFP_OK;
}

}  // namespace

extern "C" {

const char* vofp_version(void) { return "vofp 0.1 (sm_103a)"; }

vofp_status vofp_create(vofp_ctx** out, const vofp_grid* g, vofp_stream stream) {
    if (!out || !g) return VOFP_ERR_INVALID_ARG;
    *out = nullptr;
    if (g->nx <= 0 || g->ny <= 0 || g->nz <= 0 || !g->dx || !g->dy || !g->dz) return VOFP_ERR_INVALID_ARG;
    const long long n = (long long)g->nx * g->ny * g->nz;
    if (n >= (1LL << 31)) return VOFP_ERR_INVALID_ARG;
    for (int i = 0; i < g->nx; ++i)
        if (!(g->dx[i] > 0.0) || !std::isfinite(g->dx[i])) return VOFP_ERR_INVALID_ARG;
    for (int j = 0; j < g->ny; ++j)
        if (!(g->dy[j] > 0.0) || !std::isfinite(g->dy[j])) return VOFP_ERR_INVALID_ARG;
    for (int k = 0; k < g->nz; ++k)
        if (!(g->dz[k] > 0.0) || !std::isfinite(g->dz[k])) return VOFP_ERR_INVALID_ARG;
    vofp_ctx* c = new (std::nothrow) vofp_ctx();
    if (!c) return VOFP_ERR_OOM;
    c->d.nx = g->nx;
    c->d.ny = g->ny;
    c->d.nz = g->nz;
    c->d.n = n;
    c->d.plane = (long long)g->nx * g->ny;
    c->stream = reinterpret_cast<cudaStream_t>(stream);
    if (const char* e = std::getenv("VOFP_PDL")) c->pdl = std::atoi(e) != 0 ? 1 : 0;
    c->hdx.assign(g->dx, g->dx + g->nx);
    c->hdy.assign(g->dy, g->dy + g->ny);
    c->hdz.assign(g->dz, g->dz + g->nz);
    vofp_status s;
    if ((s = c->alloc(&c->dx, g->nx)) || (s = c->alloc(&c->dy, g->ny)) || (s = c->alloc(&c->dz, g->nz))) {
        vofp_destroy(c);
        return s;
    }
    if (cudaMemcpy(c->dx, g->dx, sizeof(double) * g->nx, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->dy, g->dy, sizeof(double) * g->ny, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->dz, g->dz, sizeof(double) * g->nz, cudaMemcpyHostToDevice) != cudaSuccess) {
        vofp_destroy(c);
        return VOFP_ERR_CUDA;
    }
    *out = c;
    return VOFP_OK;
}

void vofp_destroy(vofp_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    if (c->graph_fp64) cudaGraphExecDestroy(c->graph_fp64);
    if (c->graph_mixed) cudaGraphExecDestroy(c->graph_mixed);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    if (c->copy_stream) {
        cudaStreamSynchronize(c->copy_stream);
        cudaStreamDestroy(c->copy_stream);
    }
    if (c->copy_done) cudaEventDestroy(c->copy_done);
    if (c->ops_done) cudaEventDestroy(c->ops_done);
    for (cudaEvent_t e : c->set_ready)
        if (e) cudaEventDestroy(e);
    for (void* p : c->allocs) cudaFree(p);
    delete c;
}

const char* vofp_last_error(const vofp_ctx* c) { return c ? c->err.c_str() : kNullCtx; }

vofp_status vofp_build_operator(vofp_ctx* c, const double* F, const double* ax, const double* ay,
                                const double* az, const double* vf, const vofp_bc* bc, const vofp_phys* phys) {
    vofp_status s = check_ctx(c, false);
    if (s) return s;
    if (!F || !ax || !ay || !az || !bc || !phys) return invalid(c, "null input");
    for (int f = 0; f < 6; ++f)
        if (bc->kind[f] != VOFP_BC_NEUMANN && bc->kind[f] != VOFP_BC_DIRICHLET) return invalid(c, "bad boundary kind");
    if (!(phys->rho_liquid > 0.0) || !(phys->rho_gas > 0.0) || !(phys->dt > 0.0) || !(phys->merge_threshold >= 0.0) ||
        phys->merge_threshold > 1.0)
        return invalid(c, "bad physical parameters");
    // any change of the operator invalidates the captured loops (group count, pointers)
    if (c->graph_fp64) {
        cudaGraphExecDestroy(c->graph_fp64);
        c->graph_fp64 = nullptr;
        c->graph_fp64_key = -1;
    }
    if (c->graph_mixed) {
        cudaGraphExecDestroy(c->graph_mixed);
        c->graph_mixed = nullptr;
        c->graph_mixed_key = -1;
    }
    return vofp::build_operator(c, F, ax, ay, az, vf, bc, phys);
}

vofp_status vofp_rhs_from_face_velocity(vofp_ctx* c, const double* u, const double* v, const double* w,
                                        const double* body, double* b) {
    vofp_status s = check_ctx(c, true);
    if (s) return s;
    if (!u || !v || !w || !b) return invalid(c, "null input");
    if ((s = vofp::rhs(c, u, v, w, body, b))) return s;
    return fail_cuda(c);
}

vofp_status vofp_project(vofp_ctx* c, const double* p, const double* u, const double* v, const double* w,
                         const double* body, double* uo, double* vo, double* wo, double* div, double* max_div) {
    vofp_status s = check_ctx(c, true);
    if (s) return s;
    if (!p || !u || !v || !w || !uo || !vo || !wo) return invalid(c, "null input");
    if ((s = vofp::project(c, p, u, v, w, body, uo, vo, wo, div, max_div))) return s;
    return fail_cuda(c);
}

vofp_status vofp_exit_flux(vofp_ctx* c, const double* u, const double* v, const double* w, const double* body,
                           double u_c, const double* R, int balance, double* g, double* shift) {
    vofp_status s = check_ctx(c, true);
    if (s) return s;
    if (!u || (balance && (!v || !w))) return invalid(c, "null input");
    if (c->bc[1] != VOFP_BC_NEUMANN) return invalid(c, "the +x face is not NEUMANN");
    if (!std::isfinite(u_c)) return invalid(c, "u_c must be finite");
    if ((s = vofp::exit_flux(c, u, v, w, body, u_c, R, balance, g, shift))) return s;
    return fail_cuda(c);
}

vofp_status vofp_vof_flux_correct(vofp_ctx* c, const double* ax, const double* ay, const double* az,
                                  const double* u, const double* v, const double* w, double* ux_hat, double* uy_hat,
                                  double* wm_hat, double* wp_hat) {
    vofp_status s = check_ctx(c, false);
    if (s) return s;
    if (!ax || !ay || !az || !u || !v || !w || !ux_hat || !uy_hat || !wm_hat || !wp_hat)
        return invalid(c, "null input");
    if ((s = vofp::vof_flux_correct(c, ax, ay, az, u, v, w, ux_hat, uy_hat, wm_hat, wp_hat))) return s;
    return fail_cuda(c);
}

vofp_status vofp_vof_advect(vofp_ctx* c, const double* F, const double* ax, const double* ay, const double* az,
                            const double* vol_frac, const double* u, const double* v, const double* w, double dt,
                            int order, double* F_out) {
    vofp_status s = check_ctx(c, false);
    if (s) return s;
    if (!F || !ax || !ay || !az || !vol_frac || !u || !v || !w || !F_out) return invalid(c, "null input");
    if (!(dt > 0.0) || !std::isfinite(dt)) return invalid(c, "dt must be positive");
    if (order != 0 && order != 1) return invalid(c, "order must be 0 or 1");
    if ((s = vofp::vof_advect(c, F, ax, ay, az, vol_frac, u, v, w, dt, order, F_out))) return s;
    return fail_cuda(c);
}

vofp_status vofp_apply(vofp_ctx* c, const double* x, double* y) {
    vofp_status s = check_ctx(c, true);
    if (s) return s;
    if (!x || !y) return invalid(c, "null input");
    if ((s = vofp::apply_unscaled(c, x, y))) return s;
    return fail_cuda(c);
}

vofp_status vofp_residual(vofp_ctx* c, const double* b, const double* x, double* rel) {
    vofp_status s = check_ctx(c, true);
    if (s) return s;
    if (!b || !x || !rel) return invalid(c, "null input");
    return vofp::residual(c, b, x, rel);
}

vofp_status vofp_solve(vofp_ctx* c, const double* b, double* x, const vofp_solve_opts* o, vofp_solve_info* info) {
    vofp_status s = check_ctx(c, true);
    if (s) return s;
    if (!b || !x || !o) return invalid(c, "null input");
    if (!(o->rtol > 0.0) || o->rtol >= 1.0) return invalid(c, "rtol must be in (0, 1)");
    if (o->mode != VOFP_MODE_FP64 && o->mode != VOFP_MODE_MIXED && o->mode != VOFP_MODE_FCG_NN)
        return invalid(c, "unknown mode");
    if (o->mode == VOFP_MODE_FCG_NN && !o->nn) return invalid(c, "VOFP_MODE_FCG_NN needs a network");
    if (o->precond != VOFP_PRECOND_JACOBI && o->precond != VOFP_PRECOND_RBSGS) return invalid(c, "unknown preconditioner");
    if (o->check_every < 0 || (o->check_every % 2) != 0 || o->check_every > 64)
        return invalid(c, "check_every must be 0 or an even number <= 64");
    if (o->mode == VOFP_MODE_MIXED && (o->inner_rtol < 0.0 || o->inner_rtol >= 1.0))
        return invalid(c, "inner_rtol must be in [0, 1)");
    if (o->inner_restart != 0 && o->inner_restart != 1) return invalid(c, "inner_restart must be 0 or 1");
    if (o->stag_window < 0 || !(o->stag_ratio >= 0.0) || o->stag_ratio >= 1.0)
        return invalid(c, "stag_window must be >= 0 and stag_ratio in [0, 1)");
    if (info) std::memset(info, 0, sizeof(*info));
    return vofp::solve(c, b, x, o, info);
}

namespace {
// One set of a host call's inputs in device staging: cells F, vol_frac; faces ax, ay, az, u, v, w.
struct HostSet {
    double *F, *vf, *ax, *ay, *az, *u, *v, *w;
};
long long host_set_len(const vofp::Dims& d) {
    const long long nfx = (long long)(d.nx + 1) * d.ny * d.nz;
    const long long nfy = (long long)d.nx * (d.ny + 1) * d.nz;
    const long long nfz = (long long)d.nx * d.ny * (d.nz + 1);
    return 2 * d.n + 2 * (nfx + nfy + nfz);
}
HostSet host_set(const vofp::Dims& d, double* p) {
    const long long N = d.n;
    const long long nfx = (long long)(d.nx + 1) * d.ny * d.nz;
    const long long nfy = (long long)d.nx * (d.ny + 1) * d.nz;
    const long long nfz = (long long)d.nx * d.ny * (d.nz + 1);
    HostSet h;
    h.F = p;
    h.vf = p + N;
    h.ax = p + 2 * N;
    h.ay = h.ax + nfx;
    h.az = h.ay + nfy;
    h.u = h.az + nfz;
    h.v = h.u + nfx;
    h.w = h.v + nfy;
    return h;
}

// staging (b and x, then `sets` input sets), the copy stream and its events
vofp_status host_staging(vofp_ctx* c, int sets) {
    vofp_status s;
    const long long in = host_set_len(c->d);
    if (!c->dstage) {
        if ((s = c->alloc(&c->dstage, 2 * c->d.n + in))) return s;
        c->dstage_bytes += sizeof(double) * (2 * c->d.n + in);
    }
    if (sets > 1 && !c->dstage2) {
        if ((s = c->alloc(&c->dstage2, in))) return s;
        c->dstage_bytes += sizeof(double) * in;
    }
    if (!c->copy_stream) VOFP_CUDA_TRY(c, cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
    if (!c->copy_done) VOFP_CUDA_TRY(c, cudaEventCreateWithFlags(&c->copy_done, cudaEventDisableTiming));
    if (!c->ops_done) VOFP_CUDA_TRY(c, cudaEventCreateWithFlags(&c->ops_done, cudaEventDisableTiming));
    for (cudaEvent_t& e : c->set_ready)
        if (!e) VOFP_CUDA_TRY(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    return VOFP_OK;
}

// the operator's inputs (cells and apertures) and the face velocities of one step, each group on
// its own stream
vofp_status upload_ops(vofp_ctx* c, const HostSet& h, const vofp_host_step& in, cudaStream_t st) {
    const vofp::Dims d = c->d;
    const long long N = d.n;
    const long long nfx = (long long)(d.nx + 1) * d.ny * d.nz;
    const long long nfy = (long long)d.nx * (d.ny + 1) * d.nz;
    const long long nfz = (long long)d.nx * d.ny * (d.nz + 1);
    VOFP_CUDA_TRY(c, cudaMemcpyAsync(h.F, in.F, sizeof(double) * N, cudaMemcpyHostToDevice, st));
    if (in.vol_frac) VOFP_CUDA_TRY(c, cudaMemcpyAsync(h.vf, in.vol_frac, sizeof(double) * N, cudaMemcpyHostToDevice, st));
    VOFP_CUDA_TRY(c, cudaMemcpyAsync(h.ax, in.ax, sizeof(double) * nfx, cudaMemcpyHostToDevice, st));
    VOFP_CUDA_TRY(c, cudaMemcpyAsync(h.ay, in.ay, sizeof(double) * nfy, cudaMemcpyHostToDevice, st));
    VOFP_CUDA_TRY(c, cudaMemcpyAsync(h.az, in.az, sizeof(double) * nfz, cudaMemcpyHostToDevice, st));
    return VOFP_OK;
}
vofp_status upload_vel(vofp_ctx* c, const HostSet& h, const vofp_host_step& in, cudaStream_t st) {
    const vofp::Dims d = c->d;
    const long long nfx = (long long)(d.nx + 1) * d.ny * d.nz;
    const long long nfy = (long long)d.nx * (d.ny + 1) * d.nz;
    const long long nfz = (long long)d.nx * d.ny * (d.nz + 1);
    VOFP_CUDA_TRY(c, cudaMemcpyAsync(h.u, in.u, sizeof(double) * nfx, cudaMemcpyHostToDevice, st));
    VOFP_CUDA_TRY(c, cudaMemcpyAsync(h.v, in.v, sizeof(double) * nfy, cudaMemcpyHostToDevice, st));
    VOFP_CUDA_TRY(c, cudaMemcpyAsync(h.w, in.w, sizeof(double) * nfz, cudaMemcpyHostToDevice, st));
    return VOFP_OK;
}

// The steps in order. Step 0: the operator's inputs on the context stream and the face velocities
// on the copy stream, so that the velocities arrive while the operator builds. Step i + 1's inputs
// go to the other staging set on the copy stream while step i solves (that set was last read by
// step i - 1, which has finished); the copy stream starts them only after step 0's own inputs
// are in, so that they do not share the host link with the uploads step 0 waits for.
// Returns the first status other than OK (NOT_CONVERGED and BREAKDOWN go on to the next step;
// any other error ends the batch).
vofp_status solve_host_steps(vofp_ctx* c, int n, const vofp_host_step* steps, const vofp_bc* bc,
                             const vofp_phys* phys, const vofp_solve_opts* o, vofp_solve_info* infos) {
    vofp_status s = host_staging(c, n > 1 ? 2 : 1);
    if (s) return s;
    const long long N = c->d.n;
    double* db = c->dstage;
    double* dx = c->dstage + N;
    const HostSet set[2] = {host_set(c->d, c->dstage + 2 * N), host_set(c->d, n > 1 ? c->dstage2 : c->dstage + 2 * N)};
    const cudaStream_t st = c->stream, cs = c->copy_stream;
    if ((s = upload_ops(c, set[0], steps[0], st))) return s;
    VOFP_CUDA_TRY(c, cudaEventRecord(c->ops_done, st));
    if ((s = upload_vel(c, set[0], steps[0], cs))) return s;
    VOFP_CUDA_TRY(c, cudaEventRecord(c->copy_done, cs));
    if (n > 1) VOFP_CUDA_TRY(c, cudaStreamWaitEvent(cs, c->ops_done, 0));
    vofp_status first = VOFP_OK;
    for (int i = 0; i < n; ++i) {
        const HostSet& h = set[i & 1];
        if (i > 0) VOFP_CUDA_TRY(c, cudaStreamWaitEvent(st, c->set_ready[i & 1], 0));
        s = vofp_build_operator(c, h.F, h.ax, h.ay, h.az, steps[i].vol_frac ? h.vf : nullptr, bc, phys);
        if (i == 0) VOFP_CUDA_TRY(c, cudaStreamWaitEvent(st, c->copy_done, 0));
        if (s) return s;
        if ((s = vofp_rhs_from_face_velocity(c, h.u, h.v, h.w, nullptr, db))) return s;
        // the next step's uploads once this one's operator is built: the build's own small copies
        // then do not queue behind them, and the solve (kernels only) hides them
        if (i + 1 < n) {
            const HostSet& hn = set[(i + 1) & 1];
            if ((s = upload_ops(c, hn, steps[i + 1], cs)) || (s = upload_vel(c, hn, steps[i + 1], cs))) return s;
            VOFP_CUDA_TRY(c, cudaEventRecord(c->set_ready[(i + 1) & 1], cs));
        }
        vofp_solve_opts o2 = *o;
        o2.x0_zero = 1;
        const vofp_status rs = vofp_solve(c, db, dx, &o2, infos ? &infos[i] : nullptr);
        if (rs != VOFP_OK && rs != VOFP_ERR_NOT_CONVERGED && rs != VOFP_ERR_BREAKDOWN) return rs;
        VOFP_CUDA_TRY(c, cudaMemcpyAsync(steps[i].x_host, dx, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
        VOFP_CUDA_TRY(c, cudaStreamSynchronize(st));
        if (first == VOFP_OK) first = rs;
    }
    return first;
}
}  // namespace

vofp_status vofp_solve_host_batch(vofp_ctx* c, int nsteps, const vofp_host_step* steps, const vofp_bc* bc,
                                  const vofp_phys* phys, const vofp_solve_opts* o, vofp_solve_info* infos) {
    vofp_status s = check_ctx(c, false);
    if (s) return s;
    if (nsteps < 1 || !steps || !o) return invalid(c, "nsteps >= 1, steps and opts required");
    for (int i = 0; i < nsteps; ++i) {
        const vofp_host_step& h = steps[i];
        if (!h.F || !h.ax || !h.ay || !h.az || !h.u || !h.v || !h.w || !h.x_host) return invalid(c, "null input");
    }
    s = solve_host_steps(c, nsteps, steps, bc, phys, o, infos);
    // on every return the copy stream is idle: no copy still reads a caller's buffer
    if (c->copy_stream) cudaStreamSynchronize(c->copy_stream);
    return s;
}

vofp_status vofp_solve_host(vofp_ctx* c, const double* F, const double* ax, const double* ay, const double* az,
                            const double* vf, const double* u, const double* v, const double* w, const vofp_bc* bc,
                            const vofp_phys* phys, const vofp_solve_opts* o, double* x_host, vofp_solve_info* info) {
    const vofp_host_step step{F, ax, ay, az, vf, u, v, w, x_host};
    return vofp_solve_host_batch(c, 1, &step, bc, phys, o, info);
}

vofp_status vofp_scaled_pair(vofp_ctx* c, const double* b, const double* x, float* r_scaled, float* x_scaled) {
    vofp_status s = check_ctx(c, true);
    if (s) return s;
    if (!b || !x || !r_scaled || !x_scaled) return invalid(c, "null input");
    return vofp::scaled_pair(c, b, x, r_scaled, x_scaled);
}

vofp_status vofp_nn_train_step_anorm(vofp_nn* nn, vofp_ctx* c, const float* r, const float* e, float lr, int update,
                                     float* loss) {
    vofp_status s = check_ctx(c, true);
    if (s) return s;
    if (!nn || !r || !e) return invalid(c, "null input");
    return vofp::nn_train_anorm(c, nn, r, e, lr, update, loss);
}

vofp_status vofp_merge_map(vofp_ctx* c, int32_t* master) {
    vofp_status s = check_ctx(c, true);
    if (s) return s;
    if (!master) return invalid(c, "null output");
    VOFP_CUDA_TRY(c, cudaMemcpyAsync(master, c->root, sizeof(int32_t) * c->d.n, cudaMemcpyDeviceToDevice, c->stream));
    return VOFP_OK;
}

vofp_status vofp_get_stats(vofp_ctx* c, vofp_stats* st) {
    vofp_status s = check_ctx(c, true);
    if (s) return s;
    if (!st) return invalid(c, "null output");
    st->cells = c->d.n;
    st->unknowns = c->n_unknowns;
    st->inactive = c->n_inactive;
    st->merged_cells = c->n_merged;
    st->groups = c->ngroups;
    st->device_bytes = (long long)c->bytes;
    st->tma_stencil_fp32 = c->tma_ok[0] ? 1 : 0;
    st->tma_stencil_fp64 = c->tma_ok[1] ? 1 : 0;
    st->rb_compact = c->rbc_ok ? 1 : 0;
    st->pdl_chained = c->pdl ? 1 : 0;
    return VOFP_OK;
}

vofp_status vofp_launch_count(vofp_ctx* c, long long* count) {
    if (!c || !count) return VOFP_ERR_INVALID_ARG;
    *count = c->launches;
    return VOFP_OK;
}

vofp_status vofp_time_iteration_kernels(vofp_ctx* c, int precision, int precond, int reps, float* stencil_ms,
                                        float* update_ms, float* aux_ms) {
    vofp_status s = check_ctx(c, true);
    if (s) return s;
    if ((precision != 64 && precision != 32) || (precond != VOFP_PRECOND_JACOBI && precond != VOFP_PRECOND_RBSGS) ||
        reps <= 0 || !stencil_ms || !update_ms)
        return invalid(c, "bad arguments");
    float aux = 0.0f;
    s = vofp::time_iteration_kernels(c, precision, precond == VOFP_PRECOND_RBSGS, reps, stencil_ms, update_ms, &aux);
    if (aux_ms) *aux_ms = aux;
    return s;
}

}  // extern "C"
