"""GPU parity of the VOF operator (Sec. 2.4) against oracle/vof.py on the same seeded inputs.

Tolerances: the correction is the same FP64 arithmetic in the same order (1e-13 relative); after
the three stages the fractions agree to 1e-11 (the plane constants come from two root searches on
the same monotone volume, bisection in the oracle and Newton steps on the GPU, which may stop a few
units in the last place apart).
"""
import numpy as np
import pytest

from paper_1410_1937_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def vofp():
    import __graft_entry__ as g
    g.build()
    from paper_1410_1937_gb300 import vofp as V
    return V


@pytest.fixture(scope="module")
def vof():
    from oracle import vof as V
    return V


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).ravel()).cuda()


CASES = {
    "tiny16": lambda: I.tiny_sphere(n=16),
    "hull": lambda: I.config2(shape=(48, 24, 20)),
    "ragged": lambda: I.config1(shape=(36, 18, 22)),
}


def stable_dt(prob, vof, courant=0.4):
    ux, uy, wm, wp, _ = vof.flux_correct(prob)
    rate = max((np.abs(ux) / np.concatenate([prob.dx, prob.dx[-1:]])[None, None, :]).max(),
               (np.abs(uy) / np.concatenate([prob.dy, prob.dy[-1:]])[None, :, None]).max(),
               (np.maximum(np.abs(wm), np.abs(wp)) / prob.dz[:, None, None]).max())
    return courant / rate


@pytest.mark.parametrize("case", ["tiny16", "hull"])
def test_flux_correction_matches_oracle(vofp, vof, case):
    prob = CASES[case]()
    ctx = vofp.Context(prob.dx, prob.dy, prob.dz)
    t = {k: dev(getattr(prob, k)) for k in ("ax", "ay", "az", "u", "v", "w")}
    ux, uy, wm, wp = ctx.vofp_vof_flux_correct(t["ax"], t["ay"], t["az"], t["u"], t["v"], t["w"])
    rx, ry, rm, rp, _ = vof.flux_correct(prob)
    for got, ref in ((ux, rx), (uy, ry), (wm, rm), (wp, rp)):
        g = got.cpu().numpy().reshape(ref.shape)
        assert np.abs(g - ref).max() <= 1e-13 * max(np.abs(ref).max(), 1e-300)
    ctx.close()


@pytest.mark.parametrize("case", ["tiny16", "hull", "ragged"])
@pytest.mark.parametrize("order", [0, 1])
def test_advection_matches_oracle(vofp, vof, case, order):
    prob = CASES[case]()
    dt = stable_dt(prob, vof)
    ctx = vofp.Context(prob.dx, prob.dy, prob.dz)
    t = {k: dev(getattr(prob, k)) for k in ("F", "vf", "ax", "ay", "az", "u", "v", "w")}
    out = ctx.vofp_vof_advect(t["F"], t["ax"], t["ay"], t["az"], t["vf"], t["u"], t["v"], t["w"], dt, order=order)
    ref = vof.advect(prob, dt=dt, order=order)
    got = out.cpu().numpy().reshape(prob.shape)
    assert np.abs(got - ref).max() <= 1e-11
    assert np.abs(ref - prob.F).max() > 1e-3                   # the step moved the interface
    # in place (F_out = F) gives the same bits
    F2 = t["F"].clone()
    ctx.vofp_vof_advect(F2, t["ax"], t["ay"], t["az"], t["vf"], t["u"], t["v"], t["w"], dt, order=order, out=F2)
    assert torch.equal(F2, out)
    ctx.close()


def test_advection_full_size_properties(vofp, vof):
    """512 x 256 x 128 hull in waves: the step runs, stays finite and keeps cells far from the
    surface full or empty; sampled cells away from the surface against the oracle's invariant."""
    prob = I.config2()
    ctx = vofp.Context(prob.dx, prob.dy, prob.dz)
    t = {k: dev(getattr(prob, k)) for k in ("F", "vf", "ax", "ay", "az", "u", "v", "w")}
    ux, uy, wm, wp = ctx.vofp_vof_flux_correct(t["ax"], t["ay"], t["az"], t["u"], t["v"], t["w"])
    rate = max((ux.abs().max() / float(prob.dx.min())).item(), (uy.abs().max() / float(prob.dy.min())).item(),
               (torch.maximum(wm.abs(), wp.abs()).max() / float(prob.dz.min())).item())
    dt = 0.4 / rate
    out = ctx.vofp_vof_advect(t["F"], t["ax"], t["ay"], t["az"], t["vf"], t["u"], t["v"], t["w"], dt)
    torch.cuda.synchronize()
    got = out.cpu().numpy().reshape(prob.shape)
    assert np.isfinite(got).all()
    # three stages move fluid at most three cells: cells whose 7x7x7 neighbourhood is all full
    # (all empty) must stay exactly so
    from scipy.ndimage import maximum_filter, minimum_filter
    full = minimum_filter(prob.F, size=7, mode="nearest") == 1.0
    empty = maximum_filter(prob.F, size=7, mode="nearest") == 0.0
    assert full.sum() > 1000 and empty.sum() > 1000
    assert np.abs(got[full] - 1.0).max() <= 1e-12
    assert np.abs(got[empty]).max() <= 1e-12
    ctx.close()


def test_advection_small_and_degenerate_grids(vofp, vof):
    """A row of five cells with closed z faces (the oracle's one-dimensional closed form), a 7x3x5
    box of random fractions and velocities, and a single cell: GPU against the oracle."""
    z = np.zeros
    rng = np.random.default_rng(17)
    cases = []
    nx, h = 5, 0.2
    row = I.Problem(name="vof-row", dx=np.full(nx, h), dy=np.array([0.3]), dz=np.array([0.4]),
                    F=np.array([[[1.0, 1.0, 0.5, 0.0, 0.0]]]), vf=np.ones((1, 1, nx)), ax=np.ones((1, 1, nx + 1)),
                    ay=np.ones((1, 2, nx)), az=np.zeros((2, 1, nx)), u=z((1, 1, nx + 1)), v=z((1, 2, nx)),
                    w=z((2, 1, nx)))
    row.u[0, 0, :] = 0.6 * np.arange(nx + 1) * h
    cases.append((row, 0.4 * h / (0.6 * nx * h)))
    shp = (5, 3, 7)
    box = I.Problem(name="vof-box", dx=rng.uniform(0.5, 1.5, shp[2]), dy=rng.uniform(0.5, 1.5, shp[1]),
                    dz=rng.uniform(0.5, 1.5, shp[0]), F=rng.uniform(0, 1, shp), vf=np.ones(shp),
                    ax=rng.uniform(0, 1, (shp[0], shp[1], shp[2] + 1)), ay=rng.uniform(0, 1, (shp[0], shp[1] + 1, shp[2])),
                    az=rng.uniform(0, 1, (shp[0] + 1, shp[1], shp[2])), u=rng.uniform(-1, 1, (shp[0], shp[1], shp[2] + 1)),
                    v=rng.uniform(-1, 1, (shp[0], shp[1] + 1, shp[2])), w=rng.uniform(-1, 1, (shp[0] + 1, shp[1], shp[2])))
    box.F[box.F < 0.2] = 0.0
    box.F[box.F > 0.8] = 1.0
    box.vf[0, 0, 0] = 0.0
    cases.append((box, stable_dt(box, vof, 0.3)))
    one = I.Problem(name="vof-one", dx=np.array([1.0]), dy=np.array([1.0]), dz=np.array([1.0]),
                    F=np.array([[[0.3]]]), vf=np.ones((1, 1, 1)), ax=np.ones((1, 1, 2)), ay=np.ones((1, 2, 1)),
                    az=np.ones((2, 1, 1)), u=np.array([[[0.2, 0.1]]]), v=np.array([[[0.0], [0.1]]]),
                    w=np.array([[[0.1]], [[-0.2]]]))
    cases.append((one, 0.5))
    for prob, dt in cases:
        ctx = vofp.Context(prob.dx, prob.dy, prob.dz)
        t = {k: dev(getattr(prob, k)) for k in ("F", "vf", "ax", "ay", "az", "u", "v", "w")}
        for order in (0, 1):
            out = ctx.vofp_vof_advect(t["F"], t["ax"], t["ay"], t["az"], t["vf"], t["u"], t["v"], t["w"], dt,
                                      order=order)
            ref = vof.advect(prob, dt=dt, order=order)
            assert np.abs(out.cpu().numpy().reshape(prob.shape) - ref).max() <= 1e-11, (prob.name, order)
        ctx.close()
