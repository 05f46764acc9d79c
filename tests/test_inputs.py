"""The seeded input generators: structure and determinism (no GPU)."""
import numpy as np

import lp_inputs as L


def check_csr(g):
    off, idx = g.off, g.idx
    assert off[0] == 0 and off[-1] == idx.size and (np.diff(off) >= 0).all()
    src = np.repeat(np.arange(g.n), np.diff(off))
    assert (idx != src).all()                                   # no self-loops
    assert ((idx >= 0) & (idx < g.n)).all()
    for a in range(0, g.n, max(1, g.n // 200)):
        lst = idx[off[a]:off[a + 1]]
        assert (np.diff(lst) > 0).all()                         # sorted, no duplicates
    fwd = set(zip(src.tolist(), idx.tolist()))
    assert all((b, a) in fwd for a, b in list(fwd)[:5000])      # symmetric


def test_generators_structure():
    for g in (L.gnp(30, 0.2, 1), L.chung_lu(500, 10.0, 2.1, dmax=80, seed=3),
              L.rmat(10, 8, seed=2), L.grid(5, 7)):
        check_csr(g)


def test_deterministic():
    a = L.chung_lu(1000, 8.0, 2.3, dmax=100, seed=5)
    b = L.chung_lu(1000, 8.0, 2.3, dmax=100, seed=5)
    assert np.array_equal(a.off, b.off) and np.array_equal(a.idx, b.idx)
    c = L.chung_lu(1000, 8.0, 2.3, dmax=100, seed=6)
    assert not np.array_equal(a.idx, c.idx)
    r1, r2 = L.rmat(11, 4, seed=9), L.rmat(11, 4, seed=9)
    assert np.array_equal(r1.idx, r2.idx)


def test_chung_lu_shape():
    g = L.cfg_chung_lu_2k()
    assert g.n == 2000 and g.edges == 20000                     # exact top-up
    d = g.degrees()
    assert d.max() > 64                                         # hubs above the DLH limit


def test_grid_degrees():
    g = L.grid(6, 9)
    assert g.edges == 6 * 8 + 9 * 5
    d = g.degrees().reshape(6, 9)
    assert d[0, 0] == 2 and d[0, 4] == 3 and d[3, 4] == 4


def test_holdout():
    g = L.chung_lu(800, 12.0, 2.2, dmax=100, seed=8)
    s = L.holdout(g, 0.1, seed=3)
    k = int(np.floor(0.1 * g.edges))
    assert len(s.hu) == k and s.observed.edges == g.edges - k
    check_csr(s.observed)
    full = set(zip(np.repeat(np.arange(g.n), np.diff(g.off)).tolist(), g.idx.tolist()))
    obs = set(zip(np.repeat(np.arange(g.n), np.diff(s.observed.off)).tolist(),
                  s.observed.idx.tolist()))
    held = set(zip(s.hu.tolist(), s.hv.tolist()))
    assert len(held) == k and all(u < v for u, v in held)
    assert all((u, v) in full and (u, v) not in obs and (v, u) not in obs for u, v in held)
    assert obs | {(u, v) for u, v in held} | {(v, u) for u, v in held} == full
    s2 = L.holdout(g, 0.1, seed=3)
    assert np.array_equal(s.hu, s2.hu) and np.array_equal(s.hv, s2.hv)
