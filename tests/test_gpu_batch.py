"""GPU tests of the batched filter (paw_batch_create / paw_batch_cheb_filter).

Independent instances of uneven size (cells, degree, atoms, block width) run
through one captured CUDA graph.  Every instance's output must agree with a
separate paw_cheb_filter call on the same handle (same kernels; only the order
of the FP32 atomic reductions of the cell assembly differs), and, for one
instance, with the oracle's step-by-step Algorithm 2.  Replays with new
eigenvalue estimates must not recapture, and a rejected problem must leave the
other instances running.

Tolerances: FP64 is deterministic up to the assembly order (1e-12).  Two
TF32 calls on the same inputs already differ by up to ~1.5e-4 of the output
scale on these instances (the FP32 assembly order changes the rounding and the
recurrence carries it), against ~2e-3 between TF32 and FP64; 1e-3 separates
the two.
"""
import numpy as np
import pytest

import inputs
from oracle import cheb
from oracle import ops as O
from tests.gpu_util import rel_err, to_dev

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "tf32": 1e-3}
DEGREE = 6


def _systems():
    return inputs.batch_systems(count=5, n_range=(3, 4), degrees=(3, 4), atoms_range=(1, 4),
                                widths=(8, 12, 16, 20, 24), degree=DEGREE, seed=4242)


def _instances():
    import paper_2604_26037_gb300 as P
    systems = _systems()
    fes = [P.PawFE.from_system(s, block=16) for s in systems]   # B > 16: two blocks per call
    probs = []
    for k, (s, fe) in enumerate(zip(systems, fes)):
        nb = s["nvec"]
        X = to_dev(inputs.columns_of(s, range(nb)))
        tmin, up = fe.lanczos_bounds()
        lam = np.sort(np.random.default_rng(k).uniform(tmin, tmin + 0.3 * (up - tmin), nb))
        bounds = (min(lam[0], tmin) - 0.1, lam[-1] + 1e-3, up)
        probs.append([X, lam, DEGREE, bounds])
    return systems, fes, probs


def _run_batch(batch, probs, prec, lam_shift=0.0, outs=None, **kw):
    """One batched call; outs (reused between calls: pointers are part of the
    captured graph) are allocated when not given."""
    import torch
    if outs is None:
        outs = [torch.empty_like(X) for X, _, _, _ in probs]
    qs = [(X, lam + lam_shift, m, bd, out) for (X, lam, m, bd), out in zip(probs, outs)]
    st = batch.cheb_filter(qs, prec=prec, **kw)
    return st, outs


@pytest.mark.parametrize("prec", ["fp64", "tf32"])
def test_batch_matches_single_calls_and_replays(prec):
    import paper_2604_26037_gb300 as P
    systems, fes, probs = _instances()
    batch = P.PawBatch(fes, streams=3, autotune=True)
    try:
        st, outs = _run_batch(batch, probs, prec)
        assert st == [0] * len(fes)
        t0 = [batch.tuning(i) for i in range(len(fes))]
        assert all(t["captures"] >= 1 and t["graph_nodes"] > 0 for t in t0)
        assert {t["branch"] for t in t0} <= set(range(t0[0]["branches"]))
        for fe, (X, lam, m, bd), out in zip(fes, probs, outs):
            ref = fe.cheb_filter(X, lam, m, bd, prec=prec).cpu().numpy()
            assert rel_err(out.cpu().numpy(), ref) < TOL[prec]
        # replay: new eigenvalue estimates, same pointers, same graph
        ref1 = [o.cpu().numpy() for o in outs]
        st2, outs2 = _run_batch(batch, probs, prec, lam_shift=0.2, outs=outs)
        assert st2 == [0] * len(fes)
        assert batch.tuning(0)["captures"] == t0[0]["captures"]
        for fe, (X, lam, m, bd), out, r1 in zip(fes, probs, outs2, ref1):
            ref = fe.cheb_filter(X, lam + 0.2, m, bd, prec=prec).cpu().numpy()
            assert rel_err(out.cpu().numpy(), ref) < TOL[prec]
            assert rel_err(ref, r1) > 10 * TOL[prec]   # the new estimates matter at this tolerance
    finally:
        batch.close()
        for fe in fes:
            fe.close()


def test_batch_fp64_against_oracle():
    import paper_2604_26037_gb300 as P
    systems, fes, probs = _instances()
    batch = P.PawBatch(fes, streams=2, autotune=False)
    try:
        st, outs = _run_batch(batch, probs, "fp64")
        assert st == [0] * len(fes)
        k = int(np.argmin([s["ndof"] for s in systems]))
        op = O.PawOperators(systems[k])
        X, lam, m, bd = probs[k]
        ref = cheb.rchfsi_filter(op.apply_H, op.apply_S, op.apply_Sinv_approx, X.cpu().numpy(), lam, m, *bd)
        assert rel_err(outs[k].cpu().numpy(), ref) < 1e-10
    finally:
        batch.close()
        for fe in fes:
            fe.close()


def test_batch_rejected_problem_and_skipped_slot():
    import paper_2604_26037_gb300 as P
    systems, fes, probs = _instances()
    bad = list(probs[1])
    a0, bW, bU = bad[3]
    bad[3] = (bW, a0, bU)                 # a0 > bW: rejected
    probs_bad = [probs[0], bad] + probs[2:]
    batch = P.PawBatch(fes, streams=2, autotune=False)
    try:
        st, outs = _run_batch(batch, probs_bad, "tf32", raise_on_error=False)
        assert st[1] == 1                 # PAW_ERR_INVALID_ARG
        assert all(s == 0 for i, s in enumerate(st) if i != 1)
        for i in (0, 2):
            X, lam, m, bd = probs[i]
            ref = fes[i].cheb_filter(X, lam, m, bd, prec="tf32").cpu().numpy()
            assert rel_err(outs[i].cpu().numpy(), ref) < TOL["tf32"]
        # a skipped slot (None) is not an error
        import torch
        qs = [None] + [(X, lam, m, bd, torch.empty_like(X)) for X, lam, m, bd in probs[1:]]
        assert batch.cheb_filter(qs, prec="tf32") == [0] * len(fes)
    finally:
        batch.close()
        for fe in fes:
            fe.close()


def test_batch_create_rejects_repeated_handle():
    import paper_2604_26037_gb300 as P
    fe = P.PawFE.from_system(_systems()[0])
    try:
        with pytest.raises(P.PawError):
            P.PawBatch([fe, fe])
    finally:
        fe.close()
