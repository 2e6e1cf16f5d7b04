"""What the learned warm start gains: trained on solutions the multigrid computes, its
prediction (streamfunction and pressure) gives an exactly divergence-free initial guess.
Measured on held-out problems to the same absolute residual (1e-8 ||F||): the total V-cycle
count drops (the gain is small -- the 4-layer network's predictions keep 30-60% relative
error -- and no problem needs more cycles than from the zero guess).  With its two fields
rescaled to minimise ||F - K U|| the guess never starts above the zero guess's residual."""
import numpy as np
import pytest

from paper_1705_09282_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_warm_start_saves_cycles_on_held_out_problems():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_09282_gb300 import warmstart as ws
    n, p = 32, 2
    L = ws.levels_for(n)
    train = [ws.Problem(p, n, L, s, nu, seed) for (_, s, nu, seed) in inputs.batch_problems(384, 2000, sizes=(n,))]
    grids = ws.targets(train)
    net = ws.Network(seed=1)
    losses = ws.train(net, train, grids, steps=6000, batch=16, lr=3e-3)
    assert np.mean(losses[-20:]) < 0.2 * np.mean(losses[:5])
    test = [ws.Problem(p, n, L, s, nu, seed) for (_, s, nu, seed) in inputs.batch_problems(12, 9000, sizes=(n,))]
    atol = [1e-8 * float(torch.linalg.norm(pr.F)) for pr in test]
    for pr in test:
        pr.U.zero_()
    cold = ws.solve_batch_abs([pr.solver for pr in test], [pr.U for pr in test], [pr.F for pr in test], atol, 80)
    ws.predict_guesses(net, test)
    for pr in test:
        assert pr.solver.div_inf(pr.U) <= 1e-12 * max(1.0, float(pr.U.abs().max()))
    warm = ws.solve_batch_abs([pr.solver for pr in test], [pr.U for pr in test], [pr.F for pr in test], atol, 80)
    c0 = np.array([r["cycles"] for r in cold])
    c1 = np.array([r["cycles"] for r in warm])
    assert all(r["converged"] for r in cold + warm)
    print("cycles zero guess", c0.tolist(), "warm start", c1.tolist())
    assert c1.sum() < c0.sum(), (c0, c1)
    assert np.all(c1 <= c0), (c0, c1)
    assert all(r["div_inf"] <= 1e-11 for r in warm)
    # residual-minimising scaling of the same prediction: first residual <= ||F||
    ws.predict_guesses(net, test, scaled=True)
    scaled = ws.solve_batch_abs([pr.solver for pr in test], [pr.U for pr in test], [pr.F for pr in test], atol, 80)
    c2 = np.array([r["cycles"] for r in scaled])
    print("scaled warm start", c2.tolist())
    assert all(r["converged"] for r in scaled)
    for pr, r, a in zip(test, scaled, atol):
        assert r["res0"] <= (1 + 1e-9) * a / 1e-8, (r["res0"], a / 1e-8)
    assert c2.sum() <= c0.sum(), (c0, c2)
    assert all(r["div_inf"] <= 1e-11 for r in scaled)


def test_minres_scaling_recovers_a_scaled_solution():
    # the pair (alpha, beta) minimising ||F - K(alpha u + beta p)|| is (1/c, 1/c) when the
    # predicted fields are c times the exact ones (the residual then vanishes)
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_09282_gb300 import warmstart as ws
    p, n = 2, 32
    pr = ws.Problem(p, n, ws.levels_for(n), 3.0, 1.0, seed=77)
    g = ws.targets([pr])[0].clone()
    g *= 0.37
    U, a, b = ws.warm_start_minres(pr.solver, g, pr.scale, pr.p_scale, pr.F)
    # the targets are FP32 grids of an FP64 solution: agreement to their rounding
    assert abs(a * 0.37 - 1.0) < 1e-4 and abs(b * 0.37 - 1.0) < 1e-3, (a, b)
    assert pr.solver.div_inf(U) <= 1e-12 * max(1.0, float(U.abs().max()))
    # a zero prediction gives the zero guess
    U0, a0, b0 = ws.warm_start_minres(pr.solver, torch.zeros_like(g), pr.scale, pr.p_scale, pr.F)
    assert a0 == 0.0 and b0 == 0.0 and float(U0.abs().max()) == 0.0
