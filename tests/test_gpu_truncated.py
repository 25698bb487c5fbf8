"""The tree truncated at one level (wt_predict_vis_truncated), against the
CPU oracle's truncated prediction (reading R12).

* centre-snapped: each level node's pixel flux at its pixel centre, equal to
  the oracle within the mixed forms' bar (1e-6 of sum |C|);
* exact response: the same times the phase-centre pixel's exact response,
  equal to the oracle's "level" reading within the same bar;
* learned response: the network's product with the centre-snapped sum,
  within the network's own measured response error times the sum's size;
* gain at equal work: on a sky that fills the truncation level's pixels, the
  learned and exact responses are closer to the true visibilities (Eq. 12 at
  the true positions) than the centre-snapped truncation at the same level.
"""
import numpy as np
import pytest

import oracle as O
import synth

torch = pytest.importorskip("torch")
wt = pytest.importorskip("paper_1909_03956_gb300")

pytestmark = pytest.mark.gpu

RA0, DEC0 = synth.RA0, synth.DEC0
TOLMIX = 1e-6


def dev(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    return t.to(dtype) if dtype is not None else t


def _filled_sky(level, n, n_pix, seed):
    """n components uniform over a square of about n_pix x n_pix level-`level`
    pixels around the phase centre, fluxes uniform in [0.5, 1.5]."""
    rng = np.random.default_rng(seed)
    half = 0.5 * n_pix * O.level_pixel_size(level)
    return rng.uniform(-half, half, n), rng.uniform(-half, half, n), rng.uniform(0.5, 1.5, n)


@pytest.mark.parametrize("jt", [12, 10, 8, 5])
def test_snapped_truncation_matches_oracle(jt):
    w = synth.medium(n_t=4)
    J = 12
    uvw = w.uvw[::3]
    t = wt.wt_build_tree(dev(w.l), dev(w.m), dev(w.flux), w.ra0, w.dec0, J)
    got = wt.wt_predict_vis_truncated(t, jt, dev(uvw)).cpu().numpy()
    ref = O.Tree(w.l, w.m, w.flux, w.ra0, w.dec0, J).vis_truncated(jt, uvw, kind="snapped")
    assert np.max(np.abs(got - ref)) <= TOLMIX * np.abs(w.flux).sum()
    if jt == J:   # the level-J truncation is Eq. 16 (on the tensor cores for a large level)
        big = t.info()["n_leaves"] >= wt.WT_TRUNCATED_TC_MIN_NODES
        e16 = wt.wt_predict_vis(t, dev(uvw), mode=wt.WT_MIXED_TC if big else wt.WT_MIXED_FAST,
                                which=wt.WT_SUM_EQ16).cpu().numpy()
        assert np.array_equal(got, e16)


@pytest.mark.parametrize("jt,D", [(11, 3), (9, 4)])
def test_exact_response_truncation_matches_oracle(jt, D):
    w = synth.medium(n_t=4)
    uvw = w.uvw[::5]
    t = wt.wt_build_tree(dev(w.l), dev(w.m), dev(w.flux), w.ra0, w.dec0, 12)
    got = wt.wt_predict_vis_truncated(t, jt, dev(uvw), response=wt.WT_RESPONSE_EXACT, depth=D).cpu().numpy()
    ref = O.Tree(w.l, w.m, w.flux, w.ra0, w.dec0, 12).vis_truncated(jt, uvw, kind="level", depth=D)
    S = np.abs(w.flux).sum()
    assert np.max(np.abs(got - ref)) <= TOLMIX * S
    gm = wt.wt_predict_vis_truncated(t, jt, dev(uvw[:300]), response=wt.WT_RESPONSE_EXACT, depth=D,
                                     sign=-1).cpu().numpy()
    assert np.max(np.abs(gm - np.conj(ref[:300]))) <= TOLMIX * S


def _trained(level, pool, D=4, n_train=200000, steps=1500, seed=7):
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, len(pool), n_train)
    uvw = pool[idx] * np.where(rng.random((n_train, 1)) < 0.5, -1.0, 1.0)
    tgt = O.pixel_response(level, D, RA0, DEC0, uvw)
    x_max = float(np.max(np.abs(uvw * O.level_pixel_size(level)))) * 1.0001
    m = wt.Mlp(level, RA0, DEC0, depth=D, x_max=x_max, seed=seed)
    m.train(dev(uvw), dev(np.stack([tgt.real, tgt.imag], axis=1), torch.float32), steps=steps, batch=8192, lr=3e-3)
    return m


def test_learned_truncation_is_the_network_times_the_snapped_sum():
    jt, J, D = 11, 13, 4
    l, m_, f = _filled_sky(jt, 4000, 8, seed=21)
    pool = synth.medium(n_t=60).uvw
    net = _trained(jt, pool, D=D)
    uvw = pool[::max(1, len(pool) // 2000)][:2000]
    t = wt.wt_build_tree(dev(l), dev(m_), dev(f), RA0, DEC0, J)
    v_l = wt.wt_predict_vis_truncated(t, jt, dev(uvw), response=wt.WT_RESPONSE_LEARNED, mlp=net).cpu().numpy()
    snapped = wt.wt_predict_vis_truncated(t, jt, dev(uvw)).cpu().numpy()
    r_net = net.eval(dev(uvw)).cpu().numpy()
    r_ex = O.pixel_response(jt, D, RA0, DEC0, uvw)
    ref = O.Tree(l, m_, f, RA0, DEC0, J).vis_truncated(jt, uvw, kind="level", depth=D)
    S = f.sum()
    # the product itself, and the oracle within the network's response error
    assert np.max(np.abs(v_l - r_net * snapped)) <= 1e-5 * S
    assert np.all(np.abs(v_l - ref) <= np.abs(r_net - r_ex) * np.abs(snapped) + 2 * TOLMIX * S)
    with pytest.raises(wt.WtError):   # a network of another level
        wt.wt_predict_vis_truncated(t, jt - 1, dev(uvw), response=wt.WT_RESPONSE_LEARNED, mlp=net)


def test_truncation_gains_from_full_pixel_responses_at_equal_work():
    # 20 000 components filling about 8 x 8 level-11 pixels; the tree at
    # J = 13 truncated at level 11: the same level nodes, the same work per
    # visibility, three readings of what stands in a pixel
    jt, J, D = 11, 13, 4
    l, m_, f = _filled_sky(jt, 20000, 8, seed=22)
    pool = synth.medium(n_t=60).uvw
    net = _trained(jt, pool, D=D)
    uvw = pool[::max(1, len(pool) // 1500)][:1500]
    t = wt.wt_build_tree(dev(l), dev(m_), dev(f), RA0, DEC0, J)
    run = lambda resp, **kw: wt.wt_predict_vis_truncated(t, jt, dev(uvw), response=resp, **kw).cpu().numpy()
    v_true = O.dft(l, m_, f, uvw)
    rms = lambda v: float(np.sqrt(np.mean(np.abs(v - v_true) ** 2)) / f.sum())
    e_snap = rms(run(wt.WT_RESPONSE_SNAPPED))
    e_exact = rms(run(wt.WT_RESPONSE_EXACT, depth=D))
    e_learn = rms(run(wt.WT_RESPONSE_LEARNED, mlp=net))
    assert e_exact < 0.5 * e_snap, (e_exact, e_snap)
    assert e_learn < 0.8 * e_snap, (e_learn, e_snap)


@pytest.mark.parametrize("response", [wt.WT_RESPONSE_SNAPPED, wt.WT_RESPONSE_EXACT])
def test_truncation_in_both_passes(response):
    # a 20 deg field truncated at level 9 and baselines short everywhere but
    # one visibility in every 600: the level nodes' own coordinate bounds
    # decide which tiles take the grid pass and which the exact pass
    rng = np.random.default_rng(41)
    l, m_, f = rng.uniform(-0.35, 0.35, 400), rng.uniform(-0.35, 0.35, 400), 10.0 ** rng.uniform(-3, 0, 400)
    uvw = rng.uniform(-2e3, 2e3, (5000, 3))
    uvw[::600] = rng.uniform(5e4, 8e4, (len(uvw[::600]), 3)) * rng.choice([-1.0, 1.0], (len(uvw[::600]), 3))
    J, jt, D = 12, 9, 3
    t = wt.wt_build_tree(dev(l), dev(m_), dev(f), RA0, DEC0, J)
    got = wt.wt_predict_vis_truncated(t, jt, dev(uvw), response=response, depth=D).cpu().numpy()
    kind = "snapped" if response == wt.WT_RESPONSE_SNAPPED else "level"
    ref = O.Tree(l, m_, f, RA0, DEC0, J).vis_truncated(jt, uvw, kind=kind, depth=D)
    assert np.max(np.abs(got - ref)) <= TOLMIX * f.sum()
    t.close()


def test_truncation_arguments_rejected():
    w = synth.small()
    t = wt.wt_build_tree(dev(w.l), dev(w.m), dev(w.flux), w.ra0, w.dec0, 8)
    uvw = dev(w.uvw[:10])
    for bad in (dict(level=0), dict(level=9)):
        with pytest.raises(wt.WtError):
            wt.wt_predict_vis_truncated(t, bad["level"], uvw)
    with pytest.raises(wt.WtError):
        wt.wt_predict_vis_truncated(t, 5, uvw, response=wt.WT_RESPONSE_LEARNED, mlp=None)
    with pytest.raises(wt.WtError):
        wt.wt_predict_vis_truncated(t, 5, uvw, response=wt.WT_RESPONSE_EXACT, depth=9)
