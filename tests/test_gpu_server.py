"""The request server: fits and predictions served concurrently by worker
threads give the results that the same calls give one at a time, and the
oracle's: each served fit's coefficients agree with the oracle's CG on its
FP64 operator, each served prediction with the oracle's fast summation at the
oracle's coefficients (1e-5).

Each model is fitted (mixed-precision CG of Sec. 2 to tol 1e-8) and evaluated
at test points (Sec. 4.3) once through the plain entry points (krr_cg_solve,
krr_model_predict) on one stream, then again through a server where all fits
and many small prediction batches are in flight together.  The FP32 spread of the mixed operator sums with
atomics, so two runs agree to rounding, not bit for bit: predictions must match
to 1e-6 relative (the CG tolerance times the conditioning margin of these
problems), iteration counts within a refinement pass or so.
"""
import numpy as np
import pytest

import oracle
from paper_2111_10140_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2111_10140_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def problems():
    out = []
    specs = [
        (6000, 6, [(0, 1, 2), (3, 4, 5)], 0.2, 32, 6, 31),
        (9000, 4, [(0, 1), (2, 3), (1, 2)], 0.15, 32, 6, 32),
        (4000, 5, [(0, 1, 2), (2, 3), (4,)], 0.25, 32, 6, 33),
    ]
    for N, d, wins, ell, n, m, seed in specs:
        w = W.random_problem(N, d, wins, ell, n, m, seed=seed)
        w.epsB = 0.25
        rng = np.random.default_rng(seed + 100)
        Z = rng.uniform(w.X.min(0), w.X.max(0), size=(3000, d))
        out.append((w, Z))
    return out


LAM, TOL = 1.0, 1e-8


def serial_results(B, torch, probs):
    res = []
    for w, Z in probs:
        X = torch.from_numpy(w.X).cuda()
        y = torch.from_numpy(w.y).cuda()
        plan = B.anova_fastsum_plan(X, w.windows, w.ell, n=w.n, m=w.m, eps_B=w.epsB, precision=B.MIXED)
        alpha = torch.zeros_like(y)
        st, its, _ = B.krr_cg_solve(plan, LAM, y, alpha, TOL, 5000)
        # the same 500-row batches as the served predictions: a batch that
        # reaches outside the plan's ball is summed in a frame fitted to it,
        # so the approximation depends on the batch
        Zt = torch.from_numpy(Z).cuda()
        model = B.Model(plan, alpha)
        pred = torch.empty(Z.shape[0], dtype=torch.float64, device="cuda")
        plain = torch.empty_like(pred)
        for k in range(0, Z.shape[0], 500):
            model.predict(Zt[k:k + 500], pred[k:k + 500])
            B.krr_predict(plan, alpha, Zt[k:k + 500], plain[k:k + 500])
        torch.cuda.synchronize()
        res.append((int(its[0]), pred.cpu().numpy(), plain.cpu().numpy()))
        model.close()
        plan.close()
    return res


def test_server_matches_serial_calls(B, torch):
    probs = problems()
    ref = serial_results(B, torch, probs)
    sv = B.Server(n_workers=4, hbm_budget_bytes=8 << 30)
    try:
        dev = []
        for w, Z in probs:
            dev.append((torch.from_numpy(w.X).cuda(), torch.from_numpy(w.y).cuda(), torch.from_numpy(Z).cuda()))
        torch.cuda.synchronize()
        fits = [sv.submit_fit(X, w.windows, w.ell, y, LAM, n=w.n, m=w.m, eps_B=w.epsB, tol=TOL)
                for (w, _), (X, y, _) in zip(probs, dev)]
        # predictions in batches of 500 rows, interleaved over the models,
        # submitted while the fits are still running
        outs, tickets = [], []
        for k in range(6):
            for i, (_, _, Zt) in enumerate(dev):
                o = torch.full((500,), float("nan"), dtype=torch.float64, device="cuda")
                torch.cuda.synchronize()
                tickets.append((i, k, sv.submit_predict(fits[i], Zt[500 * k:500 * (k + 1)], o)))
                outs.append(o)
        fit_info = [sv.wait(t) for t in fits]
        got = [np.empty(3000) for _ in probs]
        for (i, k, t), o in zip(tickets, outs):
            r = sv.wait(t)
            assert r["status"] == B.OK
            got[i][500 * k:500 * (k + 1)] = o.cpu().numpy()
        report = []
        for (its, pred, plain), fi, g in zip(ref, fit_info, got):
            err = np.max(np.abs(g - pred)) / np.max(np.abs(pred))
            err_plain = np.max(np.abs(g - plain)) / np.max(np.abs(plain))
            report.append((fi["status"], fi["iterations"], its, err, err_plain))
        for st, it_served, it_alone, err, err_plain in report:
            assert st == B.OK, report
            # the FP32 inner passes of the refinement sum with atomics: a pass
            # may end a check interval earlier or later
            assert abs(it_served - it_alone) <= max(12, it_alone // 5), report
            assert err < 1e-6, report
            # krr_predict sums batches that leave the nodes' ball in a joint
            # frame, the model in its wide frame: two approximations within
            # the fast summation's error of each other
            assert err_plain < 1e-5, report
        # against the oracle: the served coefficients and predictions
        for i, ((w, Z), f) in enumerate(zip(probs, fits)):
            a_srv = torch.empty(w.N, dtype=torch.float64, device="cuda")
            sv.fit_alpha(f, a_srv)
            a_srv = a_srv.cpu().numpy()
            a_or, it_or, rel_or = oracle.cg(w.X, w.windows, w.eta, w.ell, w.n, w.m, LAM, w.y, TOL, 5000,
                                            sigma=w.sigma, epsB=w.epsB, p=w.p)
            assert rel_or <= TOL
            # both solve (K + lambda I) alpha = y to TOL (the GPU's FP64 operator within 1e-12 of
            # the oracle's): ||alpha_srv - alpha_or|| <= (residuals) ||y|| / lambda
            bound = (TOL + rel_or + 1e-11) * np.linalg.norm(w.y) / LAM
            assert np.linalg.norm(a_srv - a_or) <= bound, (i, np.linalg.norm(a_srv - a_or), bound)
            # predictions in the served batches against the oracle's summation at its coefficients
            ref_pred = np.concatenate([oracle.fastsum(Z[500 * k:500 * (k + 1)], w.X, w.windows, w.eta, w.ell, w.n,
                                                      w.m, a_or, sigma=w.sigma, epsB=w.epsB, p=w.p)
                                       for k in range(6)])
            assert np.linalg.norm(got[i] - ref_pred) / np.linalg.norm(ref_pred) <= 1e-5, i
        s = sv.stats()
        assert s["completed"] == len(fits) + len(tickets)
        assert 0 < s["p50_ms"] <= s["p99_ms"]
        for f in fits:
            sv.release(f)
        assert sv.stats()["bytes_in_use"] == 0
    finally:
        sv.close()


def test_server_budget_serialises_and_reports_errors(B, torch):
    """A budget below every request runs them one at a time; a fit with a bad
    window fails with EINVAL and so do predictions on it; a released model
    takes no more predictions."""
    w, Z = problems()[0]
    sv = B.Server(n_workers=3, hbm_budget_bytes=1)
    try:
        X = torch.from_numpy(w.X).cuda()
        y = torch.from_numpy(w.y).cuda()
        Zt = torch.from_numpy(Z[:700]).cuda()
        torch.cuda.synchronize()
        good = sv.submit_fit(X, w.windows, w.ell, y, LAM, n=w.n, m=w.m, eps_B=w.epsB, tol=TOL)
        bad = sv.submit_fit(X, [(0, 1, 99)], w.ell, y, LAM, m=w.m, eps_B=w.epsB, tol=TOL)
        o1 = torch.empty(700, dtype=torch.float64, device="cuda")
        o2 = torch.empty(700, dtype=torch.float64, device="cuda")
        o3 = torch.empty(700, dtype=torch.float64, device="cuda")
        t1 = sv.submit_predict(good, Zt, o1)
        t2 = sv.submit_predict(bad, Zt, o2)
        t3 = sv.submit_predict(good, Zt, o3)
        assert sv.wait(good)["status"] == B.OK
        assert sv.wait(bad)["status"] == B.EINVAL
        assert sv.wait(t1)["status"] == B.OK
        assert sv.wait(t2)["status"] == B.EINVAL
        assert sv.wait(t3)["status"] == B.OK
        assert torch.equal(o1, o3) or torch.allclose(o1, o3, rtol=0, atol=1e-12 * float(o1.abs().max()))
        sv.release(good)
        t4 = sv.submit_predict(good, Zt, o2)
        assert sv.wait(t4)["status"] == B.EINVAL
        with pytest.raises(B.AnovaError):
            sv.submit_predict(12345, Zt, o2)
        assert sv.stats()["bytes_in_use"] == 0
    finally:
        sv.close()


def test_server_fit_wait_bound_refuses_fits(B, torch):
    """With a bound on the expected queue wait, a fit submitted behind enough
    fit work is refused at once with EBUSY (nothing queued); without a bound,
    or with an empty queue, fits are admitted; predictions are never refused."""
    w, Z = problems()[1]
    sv = B.Server(n_workers=2, hbm_budget_bytes=8 << 30)
    try:
        X = torch.from_numpy(w.X).cuda()
        y = torch.from_numpy(w.y).cuda()
        torch.cuda.synchronize()
        # no bound and no measured rate yet: admitted
        f0 = sv.submit_fit(X, w.windows, w.ell, y, LAM, n=w.n, m=w.m, eps_B=w.epsB, tol=TOL)
        assert sv.wait(f0)["status"] == B.OK
        sv.set_fit_wait_bound(1e-6)
        # the queue is empty: the expected wait is 0, admitted
        f1 = sv.submit_fit(X, w.windows, w.ell, y, LAM, n=w.n, m=w.m, eps_B=w.epsB, tol=TOL)
        # behind f1 the fit would queue, and with one finished fit there is no rate yet: refused
        with pytest.raises(B.AnovaError) as e:
            sv.submit_fit(X, w.windows, w.ell, y, LAM, n=w.n, m=w.m, eps_B=w.epsB, tol=TOL)
        assert e.value.status == B.EBUSY
        Zt = torch.from_numpy(Z[:500]).cuda()
        o = torch.empty(500, dtype=torch.float64, device="cuda")
        tp = sv.submit_predict(f0, Zt, o)
        assert sv.wait(f1)["status"] == B.OK
        assert sv.wait(tp)["status"] == B.OK
        with pytest.raises(B.AnovaError):
            sv.set_fit_wait_bound(-1.0)
        sv.set_fit_wait_bound(0.0)
        f2 = sv.submit_fit(X, w.windows, w.ell, y, LAM, n=w.n, m=w.m, eps_B=w.epsB, tol=TOL)
        assert sv.wait(f2)["status"] == B.OK
        for f in (f0, f1, f2):
            sv.release(f)
        assert sv.stats()["bytes_in_use"] == 0
    finally:
        sv.close()

