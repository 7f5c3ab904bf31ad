"""Oracle pins: Philox test vectors, gamma algebra, geometry and active links.

Every check compares the oracle with something other than itself: published
test vectors, the Clifford algebra, brute-force enumeration, and the
active-link fractions the paper prints (Sec. 5: about 10% for 4^4 blocks,
8% for a 6^4 sub-block in each 8^4 block).
"""
import os

import numpy as np
import pytest

from oracle import geometry, gamma, philox, rng

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(w, 16) for w in line.split()])
    assert len(rows) == 3
    for r in rows:
        out = philox.philox4x32_10(r[0], r[1], r[2], r[3], r[4], r[5])
        assert [int(v) for v in out] == r[6:10]


def test_uniforms_and_noise_moments():
    n = 200000
    el = np.arange(n, dtype=np.uint64)
    u1, u2 = rng.uniform_pair(el, rng.PURPOSE_USER_NOISE, 3, 12345, 99)
    for u in (u1, u2):
        assert np.all((u > 0) & (u < 1))
        assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / n)
        assert abs(np.mean(u * u) - 1 / 3) < 5 * np.sqrt(4 / 45 / n)
    eta = rng.gaussian_components(el, rng.PURPOSE_USER_NOISE, 4, 12345, 99)
    # p(eta) ~ exp(-|eta|^2): E|eta|^2 = 1, E|eta|^4 = 2, E eta = 0, E eta^2 = 0
    assert abs(np.mean(np.abs(eta) ** 2) - 1) < 5 * np.sqrt(1 / n)
    assert abs(np.mean(np.abs(eta) ** 4) - 2) < 5 * np.sqrt(20 / n)
    assert abs(eta.mean()) < 5 * np.sqrt(1 / n)
    assert abs(np.mean(eta * eta)) < 5 * np.sqrt(2 / n)
    # different purposes / subs / counters give different streams
    e2 = rng.gaussian_components(el[:100], rng.PURPOSE_USER_NOISE, 5, 12345, 99)
    assert not np.allclose(e2, eta[:100])


def test_gamma_algebra():
    G = gamma.GAMMA
    for m in range(4):
        assert np.allclose(G[m], G[m].conj().T)
        for n in range(4):
            ac = G[m] @ G[n] + G[n] @ G[m]
            assert np.allclose(ac, 2 * (m == n) * np.eye(4))
    assert np.allclose(gamma.GAMMA5, np.diag([1, 1, -1, -1]))
    for m in range(4):
        assert np.allclose(gamma.GAMMA5 @ G[m], -G[m] @ gamma.GAMMA5)
    # time is lattice axis 3
    assert np.allclose(gamma.GAMMA_AXIS[3], G[0])


def test_neighbours_and_signs():
    lat = geometry.Lattice((4, 8, 2, 4), (2, 2, 2, 2))
    s = np.arange(lat.V)
    for a in range(4):
        assert np.all(lat.bwd[lat.fwd[:, a], a] == s)
        d = (lat.coords[lat.fwd[:, a]] - lat.coords) % np.array(lat.dims)
        e = np.zeros(4, dtype=int)
        e[a] = 1
        assert np.all(d == e)
    # antiperiodic sign only on hops across the time edge
    wrapf = lat.coords[:, 3] == lat.dims[3] - 1
    assert np.all(lat.sign_fwd[wrapf, 3] == -1) and np.all(lat.sign_fwd[~wrapf, 3] == 1)
    wrapb = lat.coords[:, 3] == 0
    assert np.all(lat.sign_bwd[wrapb, 3] == -1) and np.all(lat.sign_bwd[~wrapb, 3] == 1)
    assert np.all(lat.sign_fwd[:, :3] == 1)


def test_block_order_black_first():
    lat = geometry.Lattice((8, 8, 4, 4), (4, 2, 2, 2))
    order = lat.dd_order
    assert sorted(order.tolist()) == list(range(lat.V))
    col = lat.colour[order]
    assert np.all(col[: lat.n_black_sites] == 0) and np.all(col[lat.n_black_sites:] == 1)
    assert lat.n_black_sites == lat.V // 2
    # brute force: every block is contiguous, blocks in increasing id per colour,
    # sites of a block in local lexicographic order
    bid = lat.block_id[order]
    b = lat.block_sites
    for k in range(0, lat.V, b):
        assert np.all(bid[k:k + b] == bid[k])
        assert np.all(lat.local_index[order[k:k + b]] == np.arange(b))
    firsts = bid[::b]
    assert np.all(np.diff(firsts[: lat.nblocks // 2]) > 0)
    assert np.all(np.diff(firsts[lat.nblocks // 2:]) > 0)
    # face neighbours across every block face have opposite colours
    for a in range(4):
        nb = lat.fwd[:, a]
        cross = lat.block_id[nb] != lat.block_id
        assert np.all(lat.colour[nb][cross] != lat.colour[cross])


def test_active_link_fractions_printed_in_paper():
    # 4^4 blocks: 24 links per direction per block, 96 of 1024 = 9.4% ("about 10%")
    lat = geometry.Lattice((8, 8, 8, 8), (4, 4, 4, 4), active_mode="paper")
    per_block = lat.active.sum() / lat.nblocks
    assert per_block == 96
    assert np.all(lat.active.sum(axis=0) == 24 * lat.nblocks)
    assert abs(lat.active.mean() - 0.09375) < 1e-15
    # 6^4 sub-block in each 8^4 block: 1280 of 16384 = 7.8% ("8%")
    lat = geometry.Lattice((16, 16, 16, 16), (8, 8, 8, 8), active_mode="inner6")
    assert lat.active.sum() / lat.nblocks == 1280
    assert abs(lat.active.mean() - 1280 / 16384) < 1e-15
    # auto mode picks these
    assert geometry.Lattice((8, 8, 8, 8), (4, 4, 4, 4)).active_mode == "paper"
    assert geometry.Lattice((4, 4, 4, 4), (2, 2, 2, 2)).active_mode == "intra"


def _brute_force_active(lat, lo, hi):
    """Direct transcription of the rule: both ends in the region [lo, hi] of one
    block, at most one end with a nearest neighbour outside that region."""
    act = np.zeros((lat.V, 4), dtype=bool)
    for s in range(lat.V):
        def in_region(x, blk):
            return lat.block_id[x] == blk and np.all(lat.local[x] >= lo) and np.all(lat.local[x] <= hi)
        blk = lat.block_id[s]
        if not in_region(s, blk):
            continue
        def on_bnd(x):
            return any(not in_region(lat.fwd[x, a], blk) or not in_region(lat.bwd[x, a], blk) for a in range(4))
        for a in range(4):
            y = lat.fwd[s, a]
            if in_region(y, blk) and not (on_bnd(s) and on_bnd(y)):
                act[s, a] = True
    return act


def test_active_links_brute_force():
    lat = geometry.Lattice((8, 4, 4, 4), (4, 4, 2, 2), active_mode="paper")
    assert np.array_equal(lat.active, _brute_force_active(lat, 0, np.array(lat.block) - 1))
    lat = geometry.Lattice((16, 16, 8, 8), (8, 8, 8, 8), active_mode="inner6")
    assert lat.active.sum() == lat.nblocks * 1280
    assert np.array_equal(lat.active, _brute_force_active(lat, 1, np.array(lat.block) - 2))


def _plaquette_links(lat):
    s = np.arange(lat.V)
    for a in range(4):
        for b in range(a + 1, 4):
            yield [(s, a), (lat.fwd[s, a], b), (lat.fwd[s, b], a), (s, b)]


@pytest.mark.parametrize("dims,block,mode", [((8, 8, 8, 8), (4, 4, 4, 4), "paper"),
                                            ((16, 16, 8, 8), (8, 8, 4, 4), "paper"),
                                            ((16, 16, 16, 16), (8, 8, 8, 8), "inner6")])
def test_active_links_decouple(dims, block, mode):
    """No plaquette holds active links of two different blocks, so the block
    acceptance steps decouple (Sec. 3)."""
    lat = geometry.Lattice(dims, block, active_mode=mode)
    for links in _plaquette_links(lat):
        owner = np.full((lat.V, 4), -1)
        ids = []
        for (x, a) in links:
            ids.append(np.where(lat.active[x, a], lat.block_id[x], -1))
        ids = np.stack(ids, axis=1)
        for i in range(4):
            for j in range(i + 1, 4):
                both = (ids[:, i] >= 0) & (ids[:, j] >= 0)
                assert np.all(ids[both, i] == ids[both, j])


def test_intra_links_decouple_by_colour():
    """In intra mode two blocks whose links share a plaquette have opposite colours."""
    lat = geometry.Lattice((4, 4, 4, 4), (2, 2, 2, 2), active_mode="intra")
    assert lat.active.sum() == lat.nblocks * 4 * 8
    for links in _plaquette_links(lat):
        ids = np.stack([np.where(lat.active[x, a], lat.block_id[x], -1) for (x, a) in links], axis=1)
        for i in range(4):
            for j in range(i + 1, 4):
                both = (ids[:, i] >= 0) & (ids[:, j] >= 0) & (ids[:, i] != ids[:, j])
                assert np.all(lat.block_colour[ids[both, i]] != lat.block_colour[ids[both, j]])
