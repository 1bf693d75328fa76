"""The headline workload at full size (3 levels of 512 x 256, the 101-point flag, Omega_0 141 x 141, 39 762
unknowns) against the oracle on what it can compute one by one: sampled columns of B0, and the no-slip
identity after the corrector, which holds at any size (needs a GB300 and the library)."""

import numpy as np
import pytest

from oracle import grid as og
from oracle import ib as oib
from paper_2103_06415_gb300 import workloads as wl

from runners import gpu_context

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import paper_2103_06415_gb300 as p
    return p


@pytest.fixture(scope="module")
def setup():
    w = wl.flag_512x256_3lvl()
    lev = og.make_levels(w["nx"], w["ny"], w["h"], w["x0"], w["y0"], w["n_levels"])[0]
    sd = oib.Subdomain.from_box(lev, *w["sd_box"])
    return w, lev, sd


def test_sampled_b0_columns_at_full_size(lib, setup):
    """B0 of the bench's FP32 context (built in FP64 from the lattice Green's function) against the oracle's
    column solves (Eq. action) for corner, edge and interior points of Omega_0, both components."""
    w, lev, sd = setup
    ctx = gpu_context(w, precision=1)
    n2 = 2 * sd.n_sd
    assert ctx.stats()["n_sd"] == sd.n_sd
    mid = (sd.nj // 2) * sd.ni + sd.ni // 2
    for col in (0, sd.ni - 1, mid, sd.n_sd - 1, sd.n_sd + mid, n2 - 1):
        ref = oib.b0_column(sd, col, w["re"], w["dt"])
        got = ctx.operator_entries(np.arange(n2), np.full(n2, col))
        assert np.max(np.abs(got - ref)) < 1e-11 * np.max(np.abs(ref)), col
    ctx.close()


@pytest.mark.parametrize("precision,bound", [(0, 1e-10), (1, 2e-5)])
def test_no_slip_after_corrector_at_full_size(lib, setup, precision, bound):
    """After each step P E0 (C s + q_inf) equals the flag's node velocities T zeta_{n+1} (Eq. corrector2),
    with the CUDA graph the bench replays; FP32 fields bound the FP32 path's identity."""
    w, lev, sd = setup
    ctx = gpu_context(w, precision=precision)
    ctx.advance(6)
    u, v = og.faces_from_s(ctx.field(0, 1), lev)
    e0q = sd.e0(u + w["uinf"][0], v + w["uinf"][1])
    nb = w["bodies"][0]["n_pts"]
    idx, wts = ctx.interp(nb)
    ub = np.stack([(wts * e0q[idx]).sum(1), (wts * e0q[idx + sd.n_sd]).sum(1)], axis=1)
    _, zeta, _ = ctx.beam_state(0)
    vel = np.zeros((nb, 2))
    vel[1:] = zeta[:, :2]                                   # node 0 is the clamp
    scale = max(1.0, np.max(np.abs(ub)))
    assert np.max(np.abs(ub - vel)) < bound * scale
    ctx.close()


N_FULL = 12
_ORACLE = {}


def _oracle_run(w):
    """The oracle's N_FULL steps of the workload at FSI tolerance 1e-12 (computed once per module)."""
    if "sim" not in _ORACLE:
        from runners import oracle_sim
        sim = oracle_sim(w, tol=1e-12)
        for _ in range(N_FULL):
            sim.step()
        _ORACLE["sim"] = sim
    return _ORACLE["sim"]


@pytest.fixture(scope="module", params=[1, 2], ids=["shared_memory_solver", "distributed_solver"])
def full_size_runs(lib, setup, request):
    """The headline workload at full size, FP64 on the GPU (the bench's CUDA graph, the 101-CTA FSI kernel
    with owned-row assembly and the warps 0-3 barrier) and in the oracle, N_FULL steps from the same
    start, at an FSI tolerance of 1e-12 on both sides (so the iteration counts are decided far from the
    threshold and must agree)."""
    w, lev, sd = setup
    sim = _oracle_run(w)
    ctx = gpu_context(w, precision=0, tol=1e-12, fsi_solver=request.param)
    ctx.advance(N_FULL)
    nb = w["bodies"][0]["n_pts"]
    out = dict(sim=sim, hist=ctx.history(0), state=ctx.beam_state(0), interp=ctx.interp(nb),
               fields=[(ctx.field(g, 0), ctx.field(g, 1)) for g in range(w["n_levels"])])
    ctx.close()
    return out


def test_full_size_fsi_iterations_and_interpolation_map(full_size_runs):
    from runners import oracle_history
    r = full_size_runs
    ref = oracle_history(r["sim"])
    assert np.array_equal(r["hist"][:, 5], ref[:, 5])               # FSI iterations per step
    idx, wts = r["interp"]
    ridx, rw = r["sim"].last_p
    assert np.array_equal(idx, ridx)                                 # P index map bit-exact
    err = float(np.max(np.abs(wts - rw)))
    print("PARITY config2 P weights max abs %.3e" % err)
    assert err < 1e-12


def test_full_size_histories_match_oracle(full_size_runs):
    """fx, fy, tip displacement and tip rate of the flag, relative to each history's largest magnitude."""
    from runners import oracle_history, rel_err
    r = full_size_runs
    ref = oracle_history(r["sim"])
    for k, nm in ((0, "fx"), (1, "fy"), (3, "tip"), (4, "tip_rate")):
        err = rel_err(r["hist"][:, k], ref[:, k])
        print("PARITY config2 %s history rel %.3e" % (nm, err))
        assert err < 2e-11, nm


def test_full_size_flag_state_matches_oracle(full_size_runs):
    from runners import rel_err
    r = full_size_runs
    b = r["sim"].bodies[0]
    chi, zeta, zdot = r["state"]
    e_chi = float(np.max(np.abs(chi - b.chi.reshape(-1, 3))))
    e_zeta = rel_err(zeta, b.zeta.reshape(-1, 3))
    e_zdot = rel_err(zdot, b.zetadot.reshape(-1, 3))
    print("PARITY config2 chi max abs %.3e zeta rel %.3e zetadot rel %.3e" % (e_chi, e_zeta, e_zdot))
    assert e_chi < 3e-13
    assert e_zeta < 1e-10
    assert e_zdot < 1e-9


def test_full_size_fields_match_oracle(full_size_runs):
    from runners import rel_err
    r = full_size_runs
    for g, (wf, sf) in enumerate(r["fields"]):
        ew, es = rel_err(wf, r["sim"].w[g]), rel_err(sf, r["sim"].s[g])
        print("PARITY config2 level %d w rel %.3e s rel %.3e" % (g, ew, es))
        assert ew < 1e-10 and es < 1e-10, g
