"""Differentiation of a persistence loss (backward scatter kernel).

Loss = sum over the finite D0 and D2 pairs with persistence > 0.01 of
persistence squared, on tie-free Gaussian mixtures.  The analytic gradient
(dms_backward_pairs) is checked against central finite differences
(h = 1e-3) on float64 copies at 64 vertices, half drawn from the vertices
the loss depends on and half uniform; a vertex whose +-h perturbation changes
the pairing (simplices or the maximum vertices carrying their values) or the
set of pairs above the threshold is skipped (the loss is not differentiable
there); at least 16 of the 64 must remain.  The pairing the backward uses is the oracle's.
Tolerance: rtol 1e-4, atol 1e-6 (the loss is quadratic in each vertex value
for a fixed pairing, so central differences are exact up to rounding).
"""
import numpy as np
import pytest

import oracle
import synthfields as sf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ad():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2206_13932_gb300 as dms
    dms.build()
    from paper_2206_13932_gb300 import autograd
    return autograd


def _loss_and_pairs(ad, t, grid):
    dg = ad.persistence_diagram(t, grid)
    loss = ad.persistence_loss(dg, 0.01)
    keep = set()
    for d in (0, 2):
        p = (dg[d].death - dg[d].birth).detach()
        m = ((~dg[d].essential) & (p > 0.01)).cpu().numpy()
        bs = dg[d].birth_simplex.cpu().numpy()
        ds = dg[d].death_simplex.cpu().numpy()
        keep |= {(d, int(a), int(b)) for a, b, k in zip(bs, ds, m) if k}
    # the pairing, down to the maximum vertices that carry the values
    allp = set()
    for d in range(3):
        allp |= {(d, int(a), int(b), int(c), int(e)) for a, b, c, e in zip(
            dg[d].birth_simplex.cpu().numpy(), dg[d].death_simplex.cpu().numpy(),
            dg[d].birth_vertex.cpu().numpy(), dg[d].death_vertex.cpu().numpy())}
    return loss, keep, allp, dg


@pytest.mark.parametrize("edge,seed", [(24, 5001), (32, 5002)])
def test_gradient_matches_central_differences(ad, edge, seed):
    import torch
    v = sf.gaussian_mixture((edge, edge, edge), 16, seed, noise=0.0, dtype=np.float64)
    assert np.unique(v).size == v.size, "field must be tie-free"
    base = torch.from_numpy(v).cuda()
    import paper_2206_13932_gb300 as dms
    with dms.Grid((edge, edge, edge), np.float64) as grid:
        t = base.clone().requires_grad_(True)
        loss, keep, allp, dg = _loss_and_pairs(ad, t, grid)
        loss.backward()
        g = t.grad.detach().cpu().numpy().reshape(-1)
        support = np.nonzero(g)[0]
        assert support.size > 0
        rng = np.random.default_rng(seed)
        picks = list(rng.choice(support, min(32, support.size), replace=False))
        picks += list(rng.choice(v.size, 64 - len(picks), replace=False))
        h = 1e-3
        checked = 0
        for vtx in picks:
            vals = []
            ok = True
            for sgn in (1, -1):
                tp = base.clone().view(-1)
                tp[vtx] += sgn * h
                lp, kp, ap, _ = _loss_and_pairs(ad, tp.view_as(base), grid)
                if kp != keep or ap != allp:
                    ok = False
                    break
                vals.append(float(lp))
            if not ok:
                continue
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - g[vtx]) <= 1e-6 + 1e-4 * abs(fd), (vtx, fd, g[vtx])
            checked += 1
        assert checked >= 16, checked


def test_backward_pairing_is_the_oracles(ad):
    import torch
    v = sf.gaussian_mixture((14, 12, 11), 8, 77, noise=0.0, dtype=np.float64)
    t = torch.from_numpy(v).cuda()
    dg = ad.persistence_diagram(t)
    got = set()
    for d in range(3):
        got |= {(d, int(a), int(b)) for a, b in zip(dg[d].birth_simplex.cpu().numpy(),
                                                      dg[d].death_simplex.cpu().numpy())}
    want = {(int(r[0]), int(r[1]), int(r[2])) for r in oracle.pairsimplices(v)}
    assert got == want
    # births and deaths are the field's values at the maximum vertices
    flat = v.reshape(-1)
    for d in range(3):
        assert np.array_equal(dg[d].birth.detach().cpu().numpy(),
                              flat[dg[d].birth_vertex.cpu().numpy()])


def test_gradient_scatter_sums_shared_vertices(ad):
    """A vertex that is the maximum vertex of several pairs receives the sum."""
    import torch
    v = sf.white_noise((10, 9, 8), 3, np.float64)
    t = torch.from_numpy(v).cuda().requires_grad_(True)
    dg = ad.persistence_diagram(t)
    w = [torch.randn_like(dg[d].birth) for d in range(3)]
    u = [torch.randn_like(dg[d].death) for d in range(3)]
    loss = sum((dg[d].birth * w[d]).sum() + (dg[d].death * u[d]).sum() for d in range(3))
    loss.backward()
    want = np.zeros(v.size)
    for d in range(3):
        np.add.at(want, dg[d].birth_vertex.cpu().numpy(), w[d].cpu().numpy())
        fin = ~dg[d].essential.cpu().numpy()
        np.add.at(want, dg[d].death_vertex.cpu().numpy()[fin], u[d].cpu().numpy()[fin])
    assert np.allclose(t.grad.cpu().numpy().reshape(-1), want, rtol=1e-12, atol=1e-12)


def test_backward_refuses_a_newer_result(ad):
    """A grid that computed another field after the forward pass no longer
    holds the pairs the saved gradients index: the backward pass is refused
    (DMS_ERR_STATE) instead of scattering onto the new field's vertices, and
    a forward on the current result still differentiates."""
    import torch
    import paper_2206_13932_gb300 as dms
    a = sf.white_noise((10, 9, 8), 3, np.float64)
    b = sf.white_noise((10, 9, 8), 4, np.float64)      # more pairs than a's D1 for some dims
    with dms.Grid((10, 9, 8), np.float64) as g:
        ta = torch.from_numpy(a).cuda().requires_grad_(True)
        tb = torch.from_numpy(b).cuda().requires_grad_(True)
        da = ad.persistence_diagram(ta, g)          # one compute per field
        la = sum(da[d].birth.sum() for d in range(3))
        db = ad.persistence_diagram(tb, g)
        lb = sum(db[d].birth.sum() for d in range(3))
        with pytest.raises(dms.DmsError) as e:
            la.backward()
        assert e.value.status == 6
        lb.backward()
        assert tb.grad is not None and float(tb.grad.abs().sum()) > 0


def test_batch_of_eight_128_fields(ad):
    """The differentiation workload: 8 float32 128^3 mixtures (16 blobs, no
    noise, seeds 5000+i), loss summed over the batch, backward in float32,
    central differences on float64 copies of field 0.  2M float32 values
    cannot all differ; equal values are ordered by vertex id and vertices
    whose perturbation changes the pairing are skipped."""
    import torch
    import paper_2206_13932_gb300 as dms
    fields = [sf.gaussian_mixture((128, 128, 128), 16, 5000 + i, noise=0.0, dtype=np.float32)
              for i in range(8)]
    grids = [dms.Grid((128, 128, 128), np.float32) for _ in fields]
    ts = [torch.from_numpy(f).cuda().requires_grad_(True) for f in fields]
    loss = sum(ad.persistence_loss(ad.persistence_diagram(t, g), 0.01) for t, g in zip(ts, grids))
    loss.backward()
    g0 = ts[0].grad.detach().cpu().numpy().reshape(-1).astype(np.float64)
    base = torch.from_numpy(fields[0].astype(np.float64)).cuda()
    with dms.Grid((128, 128, 128), np.float64) as g64:
        l0, keep, allp, _ = _loss_and_pairs(ad, base, g64)
        rng = np.random.default_rng(5000)
        support = np.nonzero(g0)[0]
        k = min(32, support.size)
        picks = list(rng.choice(support, k, replace=False)) + list(rng.choice(g0.size, 64 - k,
                                                                            replace=False))
        h, checked = 1e-3, 0
        for vtx in picks:
            vals, ok = [], True
            for sgn in (1, -1):
                tp = base.clone().view(-1)
                tp[vtx] += sgn * h
                lp, kp, ap, _ = _loss_and_pairs(ad, tp.view_as(base), g64)
                if kp != keep or ap != allp:
                    ok = False
                    break
                vals.append(float(lp))
            if not ok:
                continue
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - g0[vtx]) <= 1e-6 + 1e-4 * abs(fd), (vtx, fd, g0[vtx])
            checked += 1
        assert checked >= 16, checked
    for g in grids:
        g.close()
