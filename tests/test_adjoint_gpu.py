"""GPU adjoint (lbm_adjoint through the C ABI) against the FP64 oracle's
adjoint, which tests/test_oracle_adjoint.py pins to finite differences, plus
GPU-side finite differences, checkpoint invariance and the autograd wrapper."""
import numpy as np
import pytest

import oracle
from paper_1710_09472_gb300 import workloads as wl
from tests.helpers import THETA, rel_linf

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_09472_gb300.build import build

    build()


# nx a multiple of 4 (and of 16 bytes per row) takes the row-staged reverse
# kernel; a ragged nx takes the general one.  "wide" rows (nx above the
# staged kernel's 256 threads) take the staged kernel with two passes per
# row and output rows of their own instead of the staged lam rows.
SHAPES = {("D2V9", "staged"): (14, 40), ("D2V9", "general"): (14, 38), ("D2V9", "wide"): (6, 320),
          ("D3V19", "staged"): (6, 7, 36), ("D3V19", "general"): (6, 7, 35), ("D3V19", "wide"): (2, 3, 288)}


def _case(vel, layout="staged"):
    shape = SHAPES[(vel, layout)]
    if vel == "D2V9":
        mask, _ = wl.boolean_obstacles(shape, 2.5, 0.8, seed=81)
        B = (0.0, 0.0, 2e-2)
    else:
        mask, _ = wl.boolean_obstacles(shape, 1.5, 0.8, seed=82)
        B = (1e-2, -2e-2, 3e-2)
    D = len(shape)
    N = mask.size
    Ef = np.zeros((D,) + shape, dtype=np.float32)
    Ef[0] = (1e-3 + 2e-4 * wl.normal(83, N)).reshape(shape)
    Ef[1] = (3e-4 * wl.normal(84, N)).reshape(shape)
    rho0 = (1.0 + 0.02 * wl.uniform01(85, N)).reshape(shape).astype(np.float32)
    u0 = (0.01 * wl.normal(86, D * N)).reshape((D,) + shape).astype(np.float32)
    wr = wl.normal(87, N).reshape(shape).astype(np.float32)
    wj = wl.normal(88, D * N).reshape((D,) + shape).astype(np.float32)
    return shape, mask, B, Ef, rho0, u0, wr, wj


def _gpu_sim(vel, shape, mask, B, Ef, rho0, u0, tau, force, storage="f32"):
    from paper_1710_09472_gb300.lbm import LBM

    sim = LBM(vel, tuple(reversed(shape)), tau, B=B, storage=storage, force=force)
    sim.set_geometry(mask.reshape(-1))
    sim.set_E_field(torch.from_numpy(Ef.reshape(-1)).cuda())
    sim.init_equilibrium(torch.from_numpy(rho0.reshape(-1)).cuda(), torch.from_numpy(u0.reshape(-1)).cuda())
    return sim


def _compare(sim, res, dE, lam0, vel, shape, mask, B, Ef, rho0, u0, wr, wj, tau, T, tb, force):
    m = oracle.Model(vel, "fd", THETA, 1.0, tau=tau, B=B, force=force)
    f0 = m.init_equilibrium(shape, mask, rho0.astype(np.float64), u0.astype(np.float64))
    states = m.trajectory(shape, mask, f0, T, Ef.astype(np.float64))
    ref = m.adjoint(shape, mask, states, tb, T, wr.astype(np.float64), wj.astype(np.float64), Ef.astype(np.float64))
    assert abs(res["loss"] / ref["loss"] - 1) < 1e-5
    gE = dE.cpu().numpy().reshape(ref["gE"].shape)
    assert rel_linf(gE, ref["gE"]) < 1e-4, rel_linf(gE, ref["gE"])
    assert rel_linf(lam0.cpu().numpy(), ref["lam0"]) < 1e-4
    comps = [2] if vel == "D2V9" else [0, 1, 2]
    for c in comps:
        assert abs(res["dL_dB"][c] - ref["gB"][c]) < 1e-4 * max(abs(ref["gB"][c]), 1e-2 * np.abs(ref["gB"]).max())
    assert abs(res["dL_dtau"] / ref["gtau"] - 1) < 1e-4


@pytest.mark.parametrize("vel", ["D2V9", "D3V19"])
@pytest.mark.parametrize("force", ["term", "shift"])
@pytest.mark.parametrize("layout", ["staged", "general", "wide"])
def test_adjoint_matches_oracle(vel, force, layout):
    shape, mask, B, Ef, rho0, u0, wr, wj = _case(vel, layout)
    tau, T, tb = 0.75, 14, 6
    sim = _gpu_sim(vel, shape, mask, B, Ef, rho0, u0, tau, force)
    D, Q, N = sim.D, sim.Q, sim.N
    dE = torch.empty(D * N, dtype=torch.float64, device="cuda")
    lam0 = torch.empty(Q * N, dtype=torch.float32, device="cuda")
    res = sim.adjoint(tb, T, torch.from_numpy(wr.reshape(-1)).cuda(), torch.from_numpy(wj.reshape(-1)).cuda(),
                      checkpoint_every=4, dL_dE=dE, dL_df0=lam0)
    _compare(sim, res, dE, lam0, vel, shape, mask, B, Ef, rho0, u0, wr, wj, tau, T, tb, force)
    sim.close()


@pytest.mark.parametrize("force", ["term", "shift"])
def test_adjoint_many_rows_porous_3d(force):
    """More rows (20 x 24 = 480) than a persistent grid has blocks, so each
    block of the row-staged reverse kernel cycles its stage ring; porous
    geometry with many bounce-back links per row."""
    shape = (20, 24, 32)
    mask, _ = wl.boolean_obstacles(shape, 2.0, 0.75, seed=97)
    B = (2e-2, -1e-2, 3e-2)
    D, N = 3, mask.size
    Ef = np.zeros((D,) + shape, dtype=np.float32)
    Ef[0] = (1e-3 + 2e-4 * wl.normal(98, N)).reshape(shape)
    Ef[2] = (3e-4 * wl.normal(99, N)).reshape(shape)
    rho0 = (1.0 + 0.02 * wl.uniform01(100, N)).reshape(shape).astype(np.float32)
    u0 = (0.01 * wl.normal(101, D * N)).reshape((D,) + shape).astype(np.float32)
    wr = wl.normal(102, N).reshape(shape).astype(np.float32)
    wj = wl.normal(103, D * N).reshape((D,) + shape).astype(np.float32)
    tau, T, tb = 0.8, 9, 3
    sim = _gpu_sim("D3V19", shape, mask, B, Ef, rho0, u0, tau, force)
    dE = torch.empty(D * N, dtype=torch.float64, device="cuda")
    lam0 = torch.empty(sim.Q * N, dtype=torch.float32, device="cuda")
    res = sim.adjoint(tb, T, torch.from_numpy(wr.reshape(-1)).cuda(), torch.from_numpy(wj.reshape(-1)).cuda(),
                      checkpoint_every=3, dL_dE=dE, dL_df0=lam0)
    _compare(sim, res, dE, lam0, "D3V19", shape, mask, B, Ef, rho0, u0, wr, wj, tau, T, tb, force)
    sim.close()
    # without dL/dE the staged reverse kernel skips the dL/dE rows; the other
    # gradients and the loss are the same numbers
    sim = _gpu_sim("D3V19", shape, mask, B, Ef, rho0, u0, tau, force)
    res2 = sim.adjoint(tb, T, torch.from_numpy(wr.reshape(-1)).cuda(), torch.from_numpy(wj.reshape(-1)).cuda(),
                       checkpoint_every=3)
    assert res2["loss"] == res["loss"] and res2["dL_dtau"] == res["dL_dtau"]
    assert np.array_equal(np.asarray(res2["dL_dB"]), np.asarray(res["dL_dB"]))
    sim.close()


def test_checkpoint_spacing_does_not_change_the_result():
    shape, mask, B, Ef, rho0, u0, wr, wj = _case("D2V9")
    outs = []
    for K in (1, 3, 0, 20):
        sim = _gpu_sim("D2V9", shape, mask, B, Ef, rho0, u0, 0.8, "term")
        dE = torch.empty(sim.D * sim.N, dtype=torch.float64, device="cuda")
        res = sim.adjoint(10, 20, wr.reshape(-1), wj.reshape(-1), checkpoint_every=K, dL_dE=dE)
        outs.append((res, dE.cpu().numpy()))
        assert sim.info()["steps"] == 20
        sim.close()
    for res, dE in outs[1:]:
        assert res["loss"] == outs[0][0]["loss"] and res["dL_dtau"] == outs[0][0]["dL_dtau"]
        assert np.array_equal(dE, outs[0][1])


@pytest.mark.parametrize("vel", ["D2V9", "D3V19"])
def test_binomial_schedule_matches_segments(vel):
    """checkpoint_every < 0 (binomial schedule with -K snapshots) and the
    budget-driven automatic choice give the same numbers, bit for bit, as the
    segment schedule: every forward state is recomputed exactly.  The forward
    step counts follow the schedules (2 T for segments; at most T (r + 1) for
    s snapshots and r sweeps with C(s + r, s) >= T)."""
    import math

    shape, mask, B, Ef, rho0, u0, wr, wj = _case(vel)
    T, tb = 23, 9
    runs = []
    for K in (5, -1, -3, -7, -40, 0, "all"):
        sim = _gpu_sim(vel, shape, mask, B, Ef, rho0, u0, 0.8, "term", storage="f16")
        if K == 0:
            # a budget below two states is refused; one of six states (the
            # segment schedule needs 5 + 4) forces the automatic choice onto
            # the binomial schedule with 4 snapshots
            state = sim.adjoint_stats()["state_bytes"]
            sim.set_memory_budget(state)
            with pytest.raises(Exception):
                sim.adjoint(tb, T, wr.reshape(-1), wj.reshape(-1), checkpoint_every=0)
            sim.close()
            sim = _gpu_sim(vel, shape, mask, B, Ef, rho0, u0, 0.8, "term", storage="f16")
            sim.set_memory_budget(6 * state)
        if K == "all":
            K = 0  # default budget: every state fits, so nothing is replayed
        dE = torch.empty(sim.D * sim.N, dtype=torch.float64, device="cuda")
        lam0 = torch.empty(sim.Q * sim.N, dtype=torch.float32, device="cuda")
        res = sim.adjoint(tb, T, wr.reshape(-1), wj.reshape(-1), checkpoint_every=K, dL_dE=dE, dL_df0=lam0)
        st = sim.adjoint_stats()
        assert sim.info()["steps"] == T and st["reverse_steps"] == T
        fT = sim.populations()
        runs.append((K, res, dE.cpu().numpy(), lam0.cpu().numpy(), fT, st))
        sim.close()
    K0, r0, e0, l0, f0, s0 = runs[0]
    assert s0["schedule"] == "segments" and s0["forward_steps"] == 2 * T - math.ceil(T / 5)
    assert runs[-1][5]["schedule"] == "store_all" and runs[-1][5]["forward_steps"] == T
    for K, res, dE, lam0, fT, st in runs[1:]:
        assert st["schedule"] in ("binomial", "store_all"), (K, st)
        if st["schedule"] == "binomial":
            s = min(-K, T) if K < 0 else 4
            r = 1
            while math.comb(s + r, s) < T:
                r += 1
            assert st["states"] == s + 2 and st["forward_steps"] <= T * (r + 1), (K, st)
        assert res["loss"] == r0["loss"] and res["dL_dtau"] == r0["dL_dtau"], K
        assert np.array_equal(np.asarray(res["dL_dB"]), np.asarray(r0["dL_dB"])), K
        assert np.array_equal(dE, e0) and np.array_equal(lam0, l0), K
        assert np.array_equal(fT, f0), K  # the context ends at the state after T steps


def test_adjoint_vs_gpu_finite_differences():
    """Central differences of the GPU forward (window totals, FP32 storage) in
    tau, B_z and the uniform E_x: relative agreement 1e-3.  (Finite differences
    of a 16-bit-stored forward measure the storage rounding, not the
    derivative; the FP16 adjoint is compared with the FP32 one instead.)"""
    storage = "f32"
    from paper_1710_09472_gb300.lbm import LBM

    shape = (32, 48)
    mask, _ = wl.boolean_obstacles(shape, 3.0, 0.75, seed=91)
    tau, E, B = 0.7, (2e-3, 5e-4), (0.0, 0.0, 5e-2)
    T, tb = 60, 40

    def loss(tau_, E_, B_):
        sim = LBM("D2V9", (48, 32), tau_, E=E_, B=B_, storage=storage, force="term")
        sim.set_geometry(mask.reshape(-1))
        sim.init_equilibrium()
        tot = sim.window_totals(tb, T)
        sim.close()
        return tot[1]  # sum over the window of the total x-current

    sim = LBM("D2V9", (48, 32), tau, E=E, B=B, storage=storage, force="term")
    sim.set_geometry(mask.reshape(-1))
    sim.init_equilibrium()
    wj = np.zeros((2, sim.N), dtype=np.float32)
    wj[0] = 1.0
    dE = torch.empty(2 * sim.N, dtype=torch.float64, device="cuda")
    res = sim.adjoint(tb, T, None, wj.reshape(-1), 0, dL_dE=dE)
    sim.close()
    gEx = float(dE.view(2, -1)[0].sum())
    h = 0.02
    fd_tau = (loss(tau * (1 + h), E, B) - loss(tau * (1 - h), E, B)) / (2 * h * tau)
    fd_B = (loss(tau, E, (0, 0, B[2] * (1 + h))) - loss(tau, E, (0, 0, B[2] * (1 - h)))) / (2 * h * B[2])
    fd_E = (loss(tau, (E[0] * (1 + h), E[1]), B) - loss(tau, (E[0] * (1 - h), E[1]), B)) / (2 * h * E[0])
    assert abs(res["dL_dtau"] / fd_tau - 1) < 1e-3, (res["dL_dtau"], fd_tau)
    assert abs(res["dL_dB"][2] / fd_B - 1) < 1e-3, (res["dL_dB"][2], fd_B)
    assert abs(gEx / fd_E - 1) < 1e-3, (gEx, fd_E)


def test_differentiable_porous_reduced_vs_oracle():
    """A 128^2 copy of the differentiable porous workload (disks r = 8,
    porosity 0.6, per-cell E_x ~ N(1e-6, 1e-7), tau = 0.7): 300 steps, loss =
    total x-current over the last 50, checkpoints every 20; per-cell dL/dE
    against the FP64 oracle adjoint."""
    w = wl.porous_2d_differentiable(n=128, steps=300)
    shape, mask, Ef = w["shape"], w["solid"], w["Efield"]
    T, tb = 300, 250
    from paper_1710_09472_gb300.lbm import LBM

    sim = LBM("D2V9", (128, 128), w["tau"], storage="f32", force="term")
    sim.set_geometry(mask.reshape(-1))
    sim.set_E_field(torch.from_numpy(Ef.reshape(-1)).cuda())
    sim.init_equilibrium()
    wj = np.zeros((2,) + shape, dtype=np.float32)
    wj[0] = 1.0
    dE = torch.empty(2 * sim.N, dtype=torch.float64, device="cuda")
    res = sim.adjoint(tb, T, None, wj.reshape(-1), 20, dL_dE=dE)
    sim.close()
    m = oracle.Model("D2V9", "fd", THETA, 1.0, tau=w["tau"], force="term")
    f0 = m.init_equilibrium(shape, mask, np.ones(shape))
    states = m.trajectory(shape, mask, f0, T, Ef.astype(np.float64))
    ref = m.adjoint(shape, mask, states, tb, T, None, wj.astype(np.float64), Ef.astype(np.float64))
    gE = dE.cpu().numpy().reshape(ref["gE"].shape)
    assert abs(res["loss"] / ref["loss"] - 1) < 1e-4
    assert rel_linf(gE, ref["gE"]) < 1e-4, rel_linf(gE, ref["gE"])


def test_autograd_function():
    from paper_1710_09472_gb300.autograd import WindowCurrent
    from paper_1710_09472_gb300.lbm import LBM

    shape = (20, 30)
    mask, _ = wl.boolean_obstacles(shape, 2.0, 0.8, seed=95)
    sim = LBM("D2V9", (30, 20), 0.8, storage="f32", force="term")
    sim.set_geometry(mask.reshape(-1))
    sim.init_equilibrium()
    E = torch.full((2,) + shape, 1e-4, dtype=torch.float32, device="cuda")
    E[1] = 0.0
    E.requires_grad_(True)
    B = torch.tensor([0.0, 0.0, 1e-2], dtype=torch.float64, requires_grad=True)
    tau = torch.tensor(0.8, dtype=torch.float64, requires_grad=True)
    J = WindowCurrent.apply(E, B, tau, sim, 20, 40, 5)
    L = J[1] + 0.5 * J[2]
    L.backward()
    # the same gradient through the library call directly
    sim2 = LBM("D2V9", (30, 20), 0.8, B=(0, 0, 1e-2), storage="f32", force="term")
    sim2.set_geometry(mask.reshape(-1))
    sim2.set_E_field(E.detach().contiguous().view(-1))
    sim2.init_equilibrium()
    wj = torch.zeros(2, sim2.N, device="cuda")
    wj[0] = 1.0
    wj[1] = 0.5
    dE = torch.empty(2 * sim2.N, dtype=torch.float64, device="cuda")
    res = sim2.adjoint(20, 40, None, wj.view(-1), 5, dL_dE=dE)
    assert torch.allclose(E.grad.double().view(-1), dE, rtol=1e-6, atol=0)
    assert abs(float(tau.grad) - res["dL_dtau"]) <= 1e-9 * abs(res["dL_dtau"])
    assert abs(float(B.grad[2]) - res["dL_dB"][2]) <= 1e-9 * abs(res["dL_dB"][2])
    sim.close()
    sim2.close()


def test_adjoint_f16_storage_close_to_f32():
    """The adjoint of an FP16-deviation-stored run agrees with the FP32-stored
    one to 1e-2 relative (the two forwards differ by the FP16 rounding)."""
    from paper_1710_09472_gb300.lbm import LBM

    shape = (32, 48)
    mask, _ = wl.boolean_obstacles(shape, 3.0, 0.75, seed=92)
    res = {}
    for storage in ("f32", "f16"):
        sim = LBM("D2V9", (48, 32), 0.7, E=(2e-3, 5e-4), B=(0, 0, 5e-2), storage=storage, force="term")
        sim.set_geometry(mask.reshape(-1))
        sim.init_equilibrium()
        wj = np.zeros((2, sim.N), dtype=np.float32)
        wj[0] = 1.0
        dE = torch.empty(2 * sim.N, dtype=torch.float64, device="cuda")
        r = sim.adjoint(40, 60, None, wj.reshape(-1), 0, dL_dE=dE)
        r["dE"] = dE.cpu().numpy()
        res[storage] = r
        sim.close()
    a, b = res["f16"], res["f32"]
    assert abs(a["dL_dtau"] / b["dL_dtau"] - 1) < 1e-2
    assert abs(a["dL_dB"][2] / b["dL_dB"][2] - 1) < 1e-2
    assert rel_linf(a["dE"], b["dE"]) < 1e-2


def test_workspace_reused_across_calls():
    """The context keeps the adjoint's buffers between calls; calls with
    different schedules on the same context (state reset in between), before
    and after lbm_release_workspace, give the same numbers bit for bit."""
    shape, mask, B, Ef, rho0, u0, wr, wj = _case("D3V19")
    T, tb = 17, 4
    sim = _gpu_sim("D3V19", shape, mask, B, Ef, rho0, u0, 0.8, "term", storage="f16")
    blob = sim.save_state()
    outs = []
    for K in (5, -3, 0, "release", 5):
        if K == "release":
            sim.release_workspace()
            continue
        sim.load_state(blob)
        dE = torch.empty(sim.D * sim.N, dtype=torch.float64, device="cuda")
        res = sim.adjoint(tb, T, wr.reshape(-1), wj.reshape(-1), checkpoint_every=K, dL_dE=dE)
        outs.append((res, dE.cpu().numpy(), sim.adjoint_stats()["schedule"]))
    assert [o[2] for o in outs] == ["segments", "binomial", "store_all", "segments"]
    for res, dE, _ in outs[1:]:
        assert res["loss"] == outs[0][0]["loss"] and res["dL_dtau"] == outs[0][0]["dL_dtau"]
        assert np.array_equal(np.asarray(res["dL_dB"]), np.asarray(outs[0][0]["dL_dB"]))
        assert np.array_equal(dE, outs[0][1])
    sim.close()
