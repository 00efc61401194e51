"""Failure detection on the GPU without a fault: a bounded device wait made
to run out, and a device allocation refused by the context's memory cap.
Both must come back as status codes, leave nothing running and leave the
context usable; the results after recovery match the oracle."""
import numpy as np
import pytest

import inputs
import oracle
from gpu_util import assert_grad_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_02991_gb300 import build
    build.build()
    import paper_2108_02991_gb300 as m
    return m


def batch(seed=11, Ns=256, shots=(24, 9, 31)):
    rng = np.random.default_rng(seed)
    Ks, grids = [], []
    for b, nc in enumerate(shots):
        K = np.cumsum(rng.normal(scale=3e-3, size=(nc, Ns, 3)), axis=1).reshape(-1, 3)
        Ks.append(np.clip(K + rng.uniform(-0.2, 0.2, size=(1, 3)), -0.45, 0.45))
        grids.append(inputs.density_gaussian(24 + 4 * b, 0.2, 0.02))
    return Ks, grids


@pytest.mark.parametrize("one_launch", [False, True])
def test_wait_budget_timeout_is_reported_and_recoverable(sp, one_launch):
    """With a zero wait budget, the batched step's projection items cannot
    wait for their trajectory's pair items (the last pair items are still
    running when the first projection item is dispensed): the step returns
    SPARKLING_E_TIMEOUT.  With the default budget restored the same context
    gives the eager result bit for bit, and that result matches the oracle's
    step."""
    Ns = 256
    Ks, grids = batch()
    K0 = np.concatenate(Ks)
    off = np.concatenate([[0], np.cumsum([k.shape[0] for k in Ks])])
    etas = [1.0 / k.shape[0] for k in Ks]
    ctx = sp.sparkling_create(0)
    try:
        rhos = [torch.from_numpy(g.rho).cuda() for g in grids]
        gs = [sp.make_grid(r, g.lo, g.hi, g.n) for r, g in zip(rhos, grids)]
        ps = [sp.make_proj(1.0 / (2 * Ns), 1.0 / (8 * Ns * Ns), 0.5, 30) for _ in Ks]

        def run():
            K = torch.from_numpy(K0).cuda()
            sp.sparkling_step_batched(ctx, K, off, Ns, gs, etas, ps, graph=False,
                                      one_launch=one_launch)
            return K

        ref = run()
        sp.sparkling_status(ctx)
        ref = ref.cpu().numpy()

        sp.sparkling_set_wait_budget(ctx, 0)
        run()
        with pytest.raises(sp.SparklingError) as e:
            sp.sparkling_status(ctx)
        assert e.value.code == sp.E_TIMEOUT, str(e.value)
        sp.sparkling_status(ctx)                      # the status word was cleared

        sp.sparkling_set_wait_budget(ctx, -1)         # the default budget again
        again = run()
        sp.sparkling_status(ctx)
        np.testing.assert_array_equal(again.cpu().numpy(), ref)
    finally:
        ctx.close()
    for b in range(len(Ks)):
        want = oracle.step(Ks[b], Ks[b].shape[0] // Ns, Ns, grids[b], etas[b], 1.0 / (2 * Ns),
                           1.0 / (8 * Ns * Ns), 0.5, -1, (0.0, 0.0, 0.0), 30)
        # the step moves by eta * G: the gradient's error bound times eta
        np.testing.assert_allclose(ref[off[b]:off[b + 1]], want, rtol=0, atol=4 * etas[b] * 1e-5)


def test_memory_cap_refuses_before_any_launch(sp):
    """A cap below the workspace a call needs gives SPARKLING_E_NOMEM before
    anything is launched; lifting it lets the same context compute the
    gradient, which matches the oracle; the host-buffer step is refused the
    same way when its device copies would pass the cap."""
    p = inputs.make_problem("tiny")
    K = torch.from_numpy(p.K).cuda()
    rho = torch.from_numpy(p.grid.rho).cuda()
    ctx = sp.sparkling_create(0)
    try:
        g = sp.make_grid(rho, p.grid.lo, p.grid.hi, p.grid.n)
        sp.sparkling_set_memory_limit(ctx, 1 << 20)
        with pytest.raises(sp.SparklingError) as e:
            sp.sparkling_grad(ctx, K, g)
        assert e.value.code == sp.E_NOMEM
        assert "limit" in str(e.value)
        assert sp.sparkling_launch_count(ctx) == 0
        sp.sparkling_set_memory_limit(ctx, 0)
        G = sp.sparkling_grad(ctx, K, g)
        sp.sparkling_status(ctx)
        _, _, G0 = oracle.forces(p.K, p.grid)
        assert_grad_close(G.cpu().numpy(), G0, "G after the cap was lifted")
        # the workspace is held now; a cap just above it refuses the extra
        # device copies of the host-buffer step
        launches = sp.sparkling_launch_count(ctx)
        sp.sparkling_set_memory_limit(ctx, 1 << 30)
        Kh = torch.from_numpy(p.K.copy())
        sp.sparkling_set_memory_limit(ctx, 1)
        pr = sp.make_proj(p.proj.alpha, p.proj.beta, p.proj.box, p.proj.n_iter)
        with pytest.raises(sp.SparklingError) as e:
            sp.sparkling_step_host(ctx, Kh, p.Nc, p.Ns, g, torch.from_numpy(p.grid.rho), p.eta, pr)
        assert e.value.code == sp.E_NOMEM
        assert sp.sparkling_launch_count(ctx) == launches
        np.testing.assert_array_equal(Kh.numpy(), p.K)
    finally:
        ctx.close()
