"""The learned planner's MLP on the GPU: forward and backward against the FP64 CPU oracle
(same BF16 rounding points), training on the cardinalities the executor logs, and what the
trained model gains over the independence heuristic it replaces."""
import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_2508_21287_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2508_21287_gb300 import build
    build.build()
    from paper_2508_21287_gb300 import binding
    return binding


def _set(B, ctx, p64):
    w = np.concatenate([p64.astype(np.float32), np.zeros(32, np.float32), np.ones(32, np.float32)])
    B.dm_model_set_weights(ctx.h, w)
    return w[:len(p64)].astype(np.float64)


@pytest.mark.parametrize("n", [16, 200, 1024])
def test_forward_backward_match_oracle(B, n):
    rng = np.random.default_rng(n)
    with B.Context(0) as ctx:
        p = _set(B, ctx, mlp.init(7))
        X = rng.normal(size=(n, 32)).astype(np.float32)
        t = rng.normal(size=n).astype(np.float32)
        pred, grads, loss = B.dm_model_grad(ctx.h, X, t)
        y_ref, loss_ref, g_ref = mlp.forward_backward(p, X.astype(np.float64), t.astype(np.float64))
        assert np.allclose(pred, y_ref, rtol=1e-3, atol=1e-3 * np.abs(y_ref).max())
        assert abs(loss - loss_ref) <= 1e-3 * loss_ref
        o = 0
        for size in mlp.SIZES:
            g, r = grads[o:o + size], g_ref[o:o + size]
            assert np.abs(g - r).max() <= 2e-2 * np.abs(r).max() + 1e-7, (o, size)
            o += size


def _log_steps(B, ctx, gid, pats, order):
    res = []
    for p in pats:
        pl = B.dm_plan(ctx.h, gid, p.n, p.row_ptr, p.col_idx, order=order)
        res.append(B.dm_match(ctx.h, pl, B.DM_COUNT))
        B.dm_plan_free(pl)
    return res


def test_training_beats_the_heuristic(B):
    g = I.heavy_hex(12, 6)
    train = [I.mixed_pattern(s, 5, 40) for s in range(1000, 1400)] + [I.sub_patch(g, 8 + s % 30, s) for s in range(200)]
    held = [I.mixed_pattern(s, 5, 40) for s in range(5000, 5120)] + [I.sub_patch(g, 8 + s % 30, 900 + s) for s in range(60)]
    with B.Context(0) as ctx:
        gid = ctx.load(g)
        B.dm_step_log(ctx.h, clear=True)
        for p in train:  # every candidate plan the learned planner weighs
            for pl in B.dm_plan_candidates(ctx.h, gid, p.n, p.row_ptr, p.col_idx):
                B.dm_match(ctx.h, pl, B.DM_COUNT)
                B.dm_plan_free(pl)
        f, t = B.dm_step_log(ctx.h, clear=True)
        assert len(t) > 1000
        B.dm_model_init(ctx.h, 3)
        losses = B.dm_model_train(ctx.h, f, t, epochs=60, batch=256, lr=2e-3, seed=3)
        print(f"{len(t)} logged steps; training MSE {losses[0]:.3f} -> {losses[-1]:.3f}")
        assert losses[-1] < 0.8 * losses[0]
        # held-out steps: the model's error against the heuristic's, on the same steps
        _log_steps(B, ctx, gid, held, B.DM_ORDER_HEURISTIC)
        fh, th = B.dm_step_log(ctx.h, clear=True)
        pred = B.dm_model_predict(ctx.h, fh)
        mae_model = float(np.mean(np.abs(pred - th)))
        mae_heur = float(np.mean(np.abs(fh[:, 22] - th)))
        print(f"held-out log-growth MAE: model {mae_model:.3f} vs heuristic {mae_heur:.3f}")
        assert mae_model < mae_heur
        # learned plans: identical results (counts and checksums) to the oracle
        got = _log_steps(B, ctx, gid, held[:40], B.DM_ORDER_LEARNED)
        for p, (c, s) in zip(held[:40], got):
            ref = oracle.enumerate(g, p, rows=False, threads=8)
            assert (c, s) == (ref.count, ref.checksum)
        # long cycles: whichever candidate the model picks, the result is the oracle's
        for n in (36, 40):
            c = I.cycle(n)
            got = _log_steps(B, ctx, gid, [c], B.DM_ORDER_LEARNED)[0]
            ref = oracle.enumerate(g, c, rows=False, threads=8)
            assert got == (ref.count, ref.checksum)
        # batched planning (host threads, one model evaluation) gives dm_plan's plans, pattern
        # by pattern, for the learned and the fixed orders
        pats = held[:60] + [I.cycle(36)]
        for order in (B.DM_ORDER_LEARNED, B.DM_ORDER_HEURISTIC, B.DM_ORDER_PAPER):
            batch = B.dm_plan_batch(ctx.h, gid, [(q.n, q.row_ptr, q.col_idx) for q in pats], order=order)
            for q, pb in zip(pats, batch):
                ps = B.dm_plan(ctx.h, gid, q.n, q.row_ptr, q.col_idx, order=order)
                assert B.dm_plan_describe(pb) == B.dm_plan_describe(ps)
                assert np.array_equal(B.dm_plan_predicted_rows(pb), B.dm_plan_predicted_rows(ps))
                B.dm_plan_free(ps)
            for q, pb in list(zip(pats, batch))[:5]:
                ref = oracle.enumerate(g, q, rows=False, threads=8)
                assert B.dm_match(ctx.h, pb, B.DM_COUNT) == (ref.count, ref.checksum)
            for pb in batch:
                B.dm_plan_free(pb)
        assert B.dm_plan_batch(ctx.h, gid, []) == []
        # a learned plan keeps the model's per-step predictions it was chosen by; a paper plan
        # keeps the independence heuristic's
        p = held[3]
        pl = B.dm_plan(ctx.h, gid, p.n, p.row_ptr, p.col_idx, order=B.DM_ORDER_LEARNED)
        f, h = B.dm_plan_estimates(pl)
        pred_plan = B.dm_model_predict(ctx.h, f).astype(np.float64)
        np.testing.assert_allclose(B.dm_plan_predicted_rows(pl), np.exp(np.cumsum(pred_plan)), rtol=1e-9)
        B.dm_plan_free(pl)
        pl = B.dm_plan(ctx.h, gid, p.n, p.row_ptr, p.col_idx)
        f, h = B.dm_plan_estimates(pl)
        np.testing.assert_allclose(B.dm_plan_predicted_rows(pl), np.exp(np.cumsum(h.astype(np.float64))), rtol=1e-9)
        B.dm_plan_free(pl)
        # checkpoint: weights out and back in give the same predictions
        w = B.dm_model_weights(ctx.h)
        B.dm_model_init(ctx.h, 99)
        B.dm_model_set_weights(ctx.h, w)
        assert np.array_equal(B.dm_model_predict(ctx.h, fh[:50]), pred[:50])
