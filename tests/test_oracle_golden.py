"""The oracle against its stored small case (tests/golden/oracle_small.json).

The stored values were written by ``tests/golden/make_golden.py`` from the oracle
alone; the paper prints no worked numeric example.  These tests are a regression
guard: a change of the oracle's arithmetic must come with a re-written case and a
commit message naming the passage of the paper that justifies it.
"""
import os
import sys

import numpy as np

import oracle
import synth

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import make_golden  # noqa: E402


def _params(d):
    return oracle.Params(K=d["K"], w_reg=d["w_reg"], eps_clip=d["eps_clip"], eps_min=d["eps_min"],
                         eps_comp=d["eps_comp"])


def test_oracle_reproduces_stored_manifold_and_gradient():
    g = make_golden.load()
    p = _params(g["params"])
    m = oracle.batch_manifold(g["geoms"], g["pair_geoms"], g["poses"], g["dims"], g["tau"], p)
    np.testing.assert_allclose(m, g["manifold"], rtol=1e-10, atol=1e-12)
    gp, gd = oracle.batch_manifold_grad(g["geoms"], g["pair_geoms"], g["poses"], g["dims"], g["tau"],
                                        g["grad_out"], p)
    np.testing.assert_allclose(gp, g["grad_poses"], rtol=1e-9, atol=1e-11)
    np.testing.assert_allclose(gd, g["grad_dims"], rtol=1e-9, atol=1e-11)


def test_stored_case_is_what_the_generators_give():
    """The stored inputs equal what make_golden builds from the seeded generators today
    (a failure here means the generators moved, not the oracle)."""
    g = make_golden.load()
    geoms, pg, poses, dims, tau, grad_out = make_golden.build_case()
    assert len(geoms) == len(g["geoms"])
    for a, b in zip(geoms, g["geoms"]):
        assert a.kind == b.kind
        for f in ("dims", "verts", "edges", "planes"):
            np.testing.assert_array_equal(np.asarray(getattr(a, f)).reshape(getattr(b, f).shape),
                                          getattr(b, f))
    for name, arr in (("pair_geoms", pg), ("poses", poses), ("dims", dims), ("tau", tau),
                      ("grad_out", grad_out)):
        np.testing.assert_array_equal(arr, g[name], err_msg=name)


def test_stored_case_structure():
    """What the case is meant to contain: every primitive kind against a hull, two
    smoothing levels, and a separated pair whose weights vanish while the rows stay finite."""
    g = make_golden.load()
    kinds = {g["geoms"][j].kind for j in g["pair_geoms"][:, 1]}
    assert set(synth.PRIMITIVE_KINDS) <= kinds | {synth.KIND_BOX}
    assert synth.KIND_HULL in {g["geoms"][j].kind for j in g["pair_geoms"][:, 0]}
    assert sorted({round(float(t), 6) for t in g["tau"]}) == [0.01, 0.1]
    m = g["manifold"]
    assert np.isfinite(m).all() and m.shape == (len(g["tau"]), g["params"]["K"], 8)
    far = m[-1]
    # every weight of the separated pair underflows, all scores -w d are ~0, so each
    # SoftSort row is uniform over the candidates and the K rows coincide
    assert far[:, 7].max() < 1e-20
    np.testing.assert_allclose(far, np.broadcast_to(far[0], far.shape), rtol=0, atol=1e-12)
    assert np.abs(m[:-1] - m[:-1, :1]).max() > 1e-3    # touching pairs: rows differ
