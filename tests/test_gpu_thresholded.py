"""Hard thresholding with full-pixel responses on the GPU
(wt_predict_vis_thresholded) against the oracle's reading T2
(oracle/threshold.py), in the reading the GPU takes: one response per
level, that of the pixel holding the phase centre ("level"), or none
("snapped").

* exact responses: equal to the oracle within the mixed forms' bar (1e-6 of
  sum |C|) for a threshold at the median |gamma|, for every coefficient kept
  and for none;
* centre-snapped: the same against the "snapped" reading;
* no coefficient kept is the tree truncated at j0, bit for bit;
* learned responses (one network per level j0 .. J): within the networks'
  own errors of the exact-response form.
"""
import numpy as np
import pytest

import oracle as O
import synth
from oracle import threshold as T

torch = pytest.importorskip("torch")
wt = pytest.importorskip("paper_1909_03956_gb300")

pytestmark = pytest.mark.gpu

TOLMIX = 1e-6
J, J0, DEPTH = 12, 9, 5          # responses on one common finest level J0 + DEPTH = J + 2


def dev(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    return t.to(dtype) if dtype is not None else t


@pytest.fixture(scope="module")
def case():
    w = synth.medium(n_t=3)
    uvw = w.uvw[::7][:2000]
    tr = O.Tree(w.l, w.m, w.flux, w.ra0, w.dec0, J)
    terms = {rd: T.full_response_terms(tr.export(), J, J0, uvw, w.ra0, w.dec0, d_leaf=DEPTH - (J - J0), reading=rd)
             for rd in ("level", "snapped")}
    t = wt.wt_build_tree(dev(w.l), dev(w.m), dev(w.flux), w.ra0, w.dec0, J)
    yield w, uvw, terms, t
    t.close()


def _level_weight_sums(w, tau):
    """Sum of |record weights| per level j0 .. J of the thresholded sum."""
    ex = O.Tree(w.l, w.m, w.flux, w.ra0, w.dec0, J).export()
    offs, lam, gam = ex["level_offsets"], ex["lam"], ex["gamma"]
    W = [float(np.sum(np.abs(T.area(J0) * lam[offs[J0 - 1]:offs[J0]])))]
    for j in range(J0, J):
        g = gam[offs[j - 1]:offs[j]]
        kept = np.where(np.abs(g) >= tau, g, 0.0)
        wc = (np.sqrt(T.area(j)) / 4.0) * kept @ T._H          # [parents][4 children]
        W.append(float(np.sum(np.abs(wc))))
    return W


def _gpu(t, uvw, tau, response, **kw):
    return wt.wt_predict_vis_thresholded(t, J0, tau, dev(uvw), response=response, **kw).cpu().numpy()


@pytest.mark.parametrize("which", ["median", "all", "none"])
@pytest.mark.parametrize("response,reading", [(wt.WT_RESPONSE_EXACT, "level"), (wt.WT_RESPONSE_SNAPPED, "snapped")])
def test_thresholded_matches_oracle(case, which, response, reading):
    w, uvw, terms, t = case
    base, G, S = terms[reading]
    tau = {"median": float(np.median(np.abs(G))), "all": 0.0, "none": float(np.max(np.abs(G))) * 2}[which]
    got = _gpu(t, uvw, tau, response, depth=DEPTH)
    ref = T.thresholded_vis_tau(base, G, S, tau)
    assert np.max(np.abs(got - ref)) <= TOLMIX * np.abs(w.flux).sum()


def test_nothing_kept_is_the_truncated_tree(case):
    w, uvw, _, t = case
    a = _gpu(t, uvw, np.inf, wt.WT_RESPONSE_EXACT, depth=DEPTH)
    b = wt.wt_predict_vis_truncated(t, J0, dev(uvw), response=wt.WT_RESPONSE_EXACT, depth=DEPTH).cpu().numpy()
    assert np.array_equal(a, b)


def test_learned_thresholded_within_the_networks_errors(case):
    w, uvw, terms, t = case
    base, G, S = terms["level"]
    tau = float(np.median(np.abs(G)))
    pool = synth.medium(n_t=60).uvw
    rng = np.random.default_rng(31)
    nets, errs = [], []
    for L in range(J0, J + 1):
        idx = rng.integers(0, len(pool), 200000)
        tu = pool[idx] * np.where(rng.random((200000, 1)) < 0.5, -1.0, 1.0)
        d = DEPTH - (L - J0)
        tg = O.pixel_response(L, d, w.ra0, w.dec0, tu)
        x_max = float(np.max(np.abs(tu * O.level_pixel_size(L)))) * 1.0001
        m = wt.Mlp(L, w.ra0, w.dec0, depth=d, x_max=x_max, seed=L)
        m.train(dev(tu), dev(np.stack([tg.real, tg.imag], axis=1), torch.float32), steps=1500, batch=8192, lr=3e-3)
        r = m.eval(dev(uvw)).cpu().numpy()
        errs.append(np.abs(r - O.pixel_response(L, d, w.ra0, w.dec0, uvw)))
        nets.append(m)
    got = _gpu(t, uvw, tau, wt.WT_RESPONSE_LEARNED, mlps=nets)
    exact = _gpu(t, uvw, tau, wt.WT_RESPONSE_EXACT, depth=DEPTH)
    # V = sum_L R_L(B) S_L(B) with |S_L| <= W_L, the level's sum of |weights|
    # (sum |F_k| at j0; below, sum over kept parents of sum_c |w_c|), so
    # |V_learned - V_exact| <= sum_L |R_net,L - R_exact,L| W_L
    W = _level_weight_sums(w, tau)
    bound = sum(e * W[i] for i, e in enumerate(errs)) + 2 * TOLMIX * np.abs(w.flux).sum()
    assert np.all(np.abs(got - exact) <= bound)
    assert np.max(np.abs(exact - T.thresholded_vis_tau(base, G, S, tau))) <= TOLMIX * np.abs(w.flux).sum()
    for m in nets:
        m.close()


def test_thresholded_arguments_rejected(case):
    w, uvw, _, t = case
    u = dev(uvw[:10])
    with pytest.raises(wt.WtError):
        wt.wt_predict_vis_thresholded(t, 0, 0.0, u)
    with pytest.raises(wt.WtError):
        wt.wt_predict_vis_thresholded(t, J0, -1.0, u)
    with pytest.raises(wt.WtError):          # the finest level must be reachable: depth >= J - j0
        wt.wt_predict_vis_thresholded(t, J0, 0.0, u, response=wt.WT_RESPONSE_EXACT, depth=J - J0 - 1)
    with pytest.raises(wt.WtError):
        wt.wt_predict_vis_thresholded(t, J0, 0.0, u, response=wt.WT_RESPONSE_LEARNED, mlps=None)
