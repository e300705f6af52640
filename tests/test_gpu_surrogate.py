"""Learned force surrogate on the GPU (tensor-core BF16 network) against the
FP64 oracle of oracle/mlp_oracle.py: forward pass, gradient, training, the
shell features of a running simulation and the forces the surrogate puts on
the particles in a step."""
import numpy as np
import pytest

from helpers import gpu_ctx, oracle_sim, rel_l2
from oracle import mlp_oracle as M
from paper_2505_10171_gb300 import workloads as W

pytestmark = pytest.mark.gpu

BF16_TOL = 2e-2  # GPU BF16 products vs the FP64 oracle on the same BF16-rounded operands


def _host():
    """A small context that hosts the network (the lattice is not used)."""
    from paper_2505_10171_gb300 import lbm
    return lbm.Context(dict(W.COMMON, nx=16, ny=16, nz=16, store_velocity=1), "fp32")


def _blocks(v):
    o = 0
    for name, shp in M.SHAPES:
        n = int(np.prod(shp))
        yield name, v[o:o + n]
        o += n


def test_forward_matches_oracle():
    th = M.init_params(8)
    X = np.random.default_rng(9).normal(size=(300, M.N_IN)).astype(np.float32)  # 3 tiles, ragged tail
    c = _host()
    c.lbm_surrogate_load(th)
    assert np.array_equal(c.lbm_surrogate_save(), th.astype(np.float32))
    Y = c.lbm_surrogate_predict(X)
    Yb, _ = M.forward(th, X, bf=True)
    Yf, _ = M.forward(th, X, bf=False)
    assert rel_l2(Y, Yb) < BF16_TOL
    assert rel_l2(Y, Yf) < 5e-2  # the BF16 rounding of the network itself
    # one row alone gives the same bits as inside the batch (no cross-row coupling)
    assert np.array_equal(c.lbm_surrogate_predict(X[137:138])[0], Y[137])
    c.close()


def test_gradient_matches_oracle():
    rng = np.random.default_rng(10)
    th = M.init_params(11) + rng.normal(scale=0.02, size=M.N_PARAM)
    th = th.astype(np.float32).astype(np.float64)
    X = rng.normal(size=(200, M.N_IN)).astype(np.float32)
    T = rng.normal(scale=0.5, size=(200, M.N_OUT)).astype(np.float32)
    c = _host()
    c.lbm_surrogate_load(th)
    g, loss = c.lbm_surrogate_gradient(X, T)
    lo, go = M.loss_and_grad(th, X, T, bf=True)
    assert abs(loss - lo) <= 5e-3 * lo
    for (name, a), (_, b) in zip(_blocks(g), _blocks(go)):
        assert rel_l2(a, b) < BF16_TOL, name
    assert np.all(M.unpack(g.astype(np.float64))["W1"][:, M.N_IN:] == 0.0)  # padding inputs
    c.close()


def test_training_follows_oracle():
    rng = np.random.default_rng(20)
    teacher = M.init_params(21)
    X = rng.normal(size=(512, M.N_IN)).astype(np.float32)
    T = M.forward(teacher, X)[0].astype(np.float32)
    th0 = M.init_params(23)
    l0 = M.loss_and_grad(th0, X, T)[0]
    c = _host()
    c.lbm_surrogate_load(th0)
    lg = c.lbm_surrogate_train(X, T, epochs=8, batch=96, lr=2e-3, seed=77)  # 96: ragged last batch
    tho, _, lo = M.train(th0, X, T, epochs=8, batch=96, lr=2e-3, seed=77, bf=True)
    assert lg < 0.5 * l0 and lo < 0.5 * l0
    assert abs(lg - lo) <= 0.1 * lo
    # the trained weights: the FP64 network's loss with them matches the oracle's
    lgw = M.loss_and_grad(c.lbm_surrogate_save().astype(np.float64), X, T)[0]
    low = M.loss_and_grad(tho, X, T)[0]
    assert abs(lgw - low) <= 0.1 * low
    c.close()


@pytest.mark.parametrize("gap,box", [(2.0, 0.0), (2.0, 8.0 / 3.0)])
def test_shell_features_match_oracle(gap, box):
    """FP64 run of the 48x32x32 drop + sphere case: the 387 inputs of the
    sphere after 20 steps against the oracle's, sampled from the oracle's own
    fields, without and with the box filter of reading c30."""
    w = W.cfg1()
    w["params"] = dict(w["params"], store_velocity=1, surrogate_shell_gap=gap, surrogate_box=box)
    steps = 20
    o = oracle_sim(w)
    o.step(steps)
    f = o.fields()
    nx, ny, nz = (w["params"][k] for k in ("nx", "ny", "nz"))
    rec = o.particles()[0]
    fo = M.shell_features(f["phi"].reshape(nz, ny, nx), f["u"].reshape(3, nz, ny, nx),
                          (o.owner() == 0).reshape(nz, ny, nx), rec[18:21], rec[21:24], rec[24:27],
                          w["particles"][0]["R"], w["particles"][0]["theta_deg"], gap, 1e-3, 8.0, box=box,
                          wall=bool(w["params"]["wall_z0"]))
    c = gpu_ctx(w, "fp64")
    c.lbm_step(steps)
    fg = c.lbm_surrogate_features()
    c.close()
    assert fg.shape == (1, M.N_IN)
    assert np.abs(fg[0] - fo).max() <= 1e-5 * max(1.0, np.abs(fo).max())
    assert np.count_nonzero(fo[0:384:4]) > 80  # most shell points have fluid corners


def test_surrogate_forces_in_the_step():
    """With the surrogate selected, the fluid force on a sphere held at rest is
    sigma R_p times the network output on its shell features (torque: sigma
    R_p^2), and the capillary share is zero."""
    from paper_2505_10171_gb300 import lbm
    w = W.cfg1()
    w["params"] = dict(w["params"], store_velocity=1)
    w["particles"] = [dict(w["particles"][0], kinematic=1)]
    th = M.init_params(31)
    c = gpu_ctx(w, "fp32")
    with pytest.raises(lbm.LbmError):
        c.lbm_set_force_model(lbm.FORCE_SURROGATE)  # no weights yet
    c.lbm_surrogate_load(th)
    c.lbm_set_force_model(lbm.FORCE_SURROGATE)
    c.lbm_step(6)
    rec = c.lbm_particle_forces()[0]
    y = c.lbm_surrogate_predict(c.lbm_surrogate_features())[0].astype(np.float64)
    sR = w["params"]["sigma"] * w["particles"][0]["R"]
    assert np.allclose(rec[0:3], sR * y[0:3], rtol=1e-6, atol=0)
    assert np.allclose(rec[3:6], sR * w["particles"][0]["R"] * y[3:6], rtol=1e-6, atol=0)
    assert np.all(rec[6:12] == 0.0)
    c.lbm_set_force_model(lbm.FORCE_RESOLVED)
    c.lbm_step(1)
    assert np.any(c.lbm_particle_forces()[0][6:12] != 0.0)  # the resolved capillary force is back
    c.close()


def test_coarse_campaign_pipeline():
    """The training and evaluation campaign end to end on a small scale: two
    resolved training runs paired with their coarse runs and one held-out
    set-up, 640 steps.  The training loss falls, every error is finite, and
    with the spheres held the in-loop surrogate forces equal the network's
    offline predictions on the plain coarse run's inputs."""
    from paper_2505_10171_gb300 import surrogate_study as SS
    table, rec = SS.campaign([1, 2], [101], steps=640, every=32, epochs=6, win=4)
    print(table)
    assert table["samples"] == 2 * 20 * 8
    assert rec["losses"][-1] < rec["losses"][0]
    for k in ("offline_raw", "plain_coarse_raw", "surrogate_coarse_raw", "offline_smoothed"):
        assert np.all(np.isfinite(table[k]))
    assert np.allclose(table["offline_raw"], table["surrogate_coarse_raw"], rtol=1e-6)


def test_trained_surrogate_beats_plain_coarse_forces():
    """What the trained network gains: the campaign's weights (trained on
    2 x 10^5 paired samples of 25 seeds, committed with the campaign's record)
    on two seeds outside its training and evaluation sets.  In the coarse
    96x48x48 runs (R_p = 3) the surrogate's force error against the resolved
    R_p = 8 runs at matched steps is below the plain coarse method's, over all
    samples and over those where a sphere touches the drop."""
    import os
    from paper_2505_10171_gb300 import surrogate_study as SS
    path = os.path.join(os.path.dirname(SS.__file__), "records", "surrogate_weights_96x48x48.npy")
    weights = np.load(path)
    seeds, steps, every = [2001, 2002], 16000, 16
    ref = SS.run([SS.resolved(s) for s in seeds], steps, every, features=False)
    plain = SS.run([SS.coarse(s) for s in seeds], steps, every)
    sur = SS.run([SS.coarse(s) for s in seeds], steps, every, weights=weights, features=False)
    Yr = np.concatenate([r["Y"] for r in ref])
    Yp = np.concatenate([r["Y"] for r in plain])
    Ys = np.concatenate([r["Y"] for r in sur])
    touch = np.concatenate([SS.touching(r["X"]) for r in plain])
    e_plain, e_sur = SS.errors(Yp, Yr)[0], SS.errors(Ys, Yr)[0]
    t_plain, t_sur = SS.errors(Yp, Yr, touch)[0], SS.errors(Ys, Yr, touch)[0]
    print(dict(all=(e_sur, e_plain), touching=(t_sur, t_plain), touching_fraction=float(touch.mean())))
    assert touch.mean() > 0.05  # the drop sweeps over some of the spheres
    assert e_sur < 0.9 * e_plain
    assert t_sur < 0.9 * t_plain


def test_bounded_wait_gives_up_and_reports_timeout():
    """The failure path of the tensor-core GEMM's bounded wait, with no device
    fault: under the host-set injection the GEMM issues no MMA and never
    signals its commit barrier, the wait runs out, the kernel frees its tensor
    memory and returns, and the call reports LBM_ERR_TIMEOUT.  The GPU stays
    usable: a fresh context computes the same forward pass as before."""
    from paper_2505_10171_gb300 import lbm
    th = M.init_params(8)
    X = np.random.default_rng(3).normal(size=(150, M.N_IN)).astype(np.float32)
    c = _host()
    c.lbm_surrogate_load(th)
    Y0 = c.lbm_surrogate_predict(X)
    c.lbm_inject_fault(lbm.FAULT_GEMM_NO_COMMIT)
    with pytest.raises(lbm.LbmError) as e:
        c.lbm_surrogate_predict(X)
    assert e.value.status == lbm.LBM_ERR_TIMEOUT
    with pytest.raises(lbm.LbmError) as e:
        c.lbm_inject_fault(7)
    assert e.value.status == lbm.LBM_ERR_ARG
    c.close()
    c = _host()
    c.lbm_surrogate_load(th)
    assert np.array_equal(c.lbm_surrogate_predict(X), Y0)
    c.close()
