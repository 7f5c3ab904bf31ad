"""Host-side logic of the library that needs no GPU: the division-by-
multiplication rule of the index arithmetic, the block-order position of a
block, and the workspace planning through the C ABI's size query."""
import ctypes
import random

import numpy as np

from oracle import geometry


def fast_div_magic(d, vh):
    """ceil(2^32 / d) when every dividend below vh satisfies n * d < 2^32."""
    if d <= 1 or vh * d >= 2 ** 32:
        return 0
    return ((1 << 32) + d - 1) // d


def test_fast_division_is_exact_where_enabled():
    rs = random.Random(1)
    for d in range(2, 130):
        for vh in (2 ** 10, 2 ** 20, 3 * 2 ** 19, 2 ** 23):
            m = fast_div_magic(d, vh)
            if not m:
                continue
            ns = list(range(0, min(vh, 20000))) + [rs.randrange(vh) for _ in range(20000)] + [vh - 1]
            for n in ns:
                assert (n * m) >> 32 == n // d, (d, vh, n)


def block_pos_to_id(pos, nbk):
    """Host mirror of the block-order rule: blocks of one colour in
    increasing id, black first; position -> block id."""
    nb = int(np.prod(nbk))
    half = nb // 2
    col = 1 if pos >= half else 0
    rank = pos - col * half
    bid = 2 * rank
    b1 = (bid // nbk[0]) % nbk[1]
    b2 = (bid // (nbk[0] * nbk[1])) % nbk[2]
    b3 = bid // (nbk[0] * nbk[1] * nbk[2])
    if (b1 + b2 + b3) % 2 != col:
        bid += 1
    return bid


def test_block_position_rule_matches_block_order():
    for dims, block in [((8, 8, 8, 8), (4, 4, 4, 4)), ((32, 32, 32, 64), (8, 8, 8, 8)),
                        ((16, 8, 12, 4), (4, 2, 6, 2))]:
        lat = geometry.Lattice(dims, block)
        firsts = lat.block_id[lat.dd_order[:: lat.block_sites]]
        got = [block_pos_to_id(p, lat.nblock_dims) for p in range(lat.nblocks)]
        assert got == list(firsts)


def test_workspace_size_query_without_gpu():
    """dd_init needs a device; the size rule itself is exercised on the GPU.
    Here: the binding's parameter struct has the fields of the header's
    dd_params, in the header's order."""
    import os
    import re
    from paper_1112_1243_gb300 import _lib
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "dd.h")).read()
    body = re.search(r"typedef struct \{(.*?)\} dd_params;", hdr, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    declared = re.findall(r"\b(?:int|double)\s+(\w+)", body)
    names = [f[0] for f in _lib.dd_params._fields_]
    assert names == declared and "sap_nkv" in names
    assert ctypes.sizeof(_lib.dd_params) % 8 == 0


def test_variance_fits_and_acceptance():
    """Host-side analysis of the 1/N extrapolation: exact data are fitted
    exactly, and the acceptance formula agrees with the oracle's statement of
    the Gaussian law."""
    from oracle import accept
    from paper_1112_1243_gb300 import variance
    Ns = [1, 2, 4, 8, 16]
    a, b = variance.fit_inverse_n(Ns, [0.7 + 2.5 / n for n in Ns])
    assert abs(a - 0.7) < 1e-12 and abs(b - 2.5) < 1e-12
    assert abs(variance.fit_through_zero([1, 2, 3], [2.0, 4.0, 6.0]) - 2.0) < 1e-12
    for s2 in (0.0, 0.3, 1.0, 4.0, 25.0):
        assert abs(variance.exact_acceptance(s2) - accept.gaussian_acceptance(s2)) < 1e-15


def test_roofline_entries():
    """Roofline entries of the benchmark from timed units and milliseconds:
    HBM kinds in GB/s against the copy bandwidth, ALU kinds in TFLOP/s
    against the pipe's peak; the Dirichlet kinds count only the hops that
    stay inside a block (7 of 8 for 8^4 blocks)."""
    import bench
    assert abs(bench.hops_kept((8, 8, 8, 8)) - 7.0) < 1e-15
    assert abs(bench.hops_kept((4, 4, 4, 4)) - 6.0) < 1e-15
    m = bench.kernel_models((8, 8, 8, 8))
    alu = {"fp64_fma": 1.25, "fp32_fma": 78.0}
    r = bench.roofline_entry(2, m[2], 23.0, 10, 12 * 1048576, 2300.0, 6800.0, alu, "probe")
    assert r["bound"] == "alu" and r["unit_rate"] == "TFLOP/s" and r["pipe"] == "fp64_fma"
    assert abs(r["achieved"] - 12 * 1048576 * 1368 / 0.023 / 1e12) < 1e-12
    assert abs(r["frac"] - r["achieved"] / 1.25) < 1e-15
    assert abs(r["share_of_step"] - 23.0 / 2300.0) < 1e-15
    r4 = bench.roofline_entry(4, m[4], 10.0, 4, 1000, 100.0, 6800.0, alu, "probe")
    assert r4["flops_per_unit"] == 48 + 165 * 7 and r4["bound"] == "alu"
    r1 = bench.roofline_entry(1, m[1], 1.0, 1, 1e6, 100.0, 6800.0, alu, "probe")
    assert r1["bound"] == "hbm" and abs(r1["achieved"] - 1e6 * 436 / 1e9 / 1e-3) < 1e-9
    assert abs(r1["frac"] - r1["achieved"] / 6800.0) < 1e-15
    assert bench.roofline_entry(2, m[2], 0.0, 1, 10, 1.0, 6800.0, alu, "probe") is None
    assert bench.roofline_entry(2, m[2], 1.0, 1, 0, 1.0, 6800.0, alu, "probe") is None


def colour_site(L, b, c, t, p):
    """The arithmetic the hop kernels use for the t-th site of the blocks of
    colour c (even block extent along axis 0): even-odd index h and x."""
    Lh0 = L[0] // 2
    q = Lh0 // 2
    r, u = divmod(t, q)
    B = b[0] // 2
    m, k = divmod(u, B)
    x1 = r % L[1]
    x2 = (r // L[1]) % L[2]
    x3 = r // (L[1] * L[2])
    cr = (x1 // b[1] + x2 // b[2] + x3 // b[3]) & 1
    hx = (2 * m + ((c + cr) & 1)) * B + k
    x0 = 2 * hx + ((p + x1 + x2 + x3) & 1)
    return hx + Lh0 * r, (x0, x1, x2, x3)


def test_colour_site_arithmetic_lists_the_colour_sets():
    """For every parity, the computed sites are the sites of the blocks of
    colour c (colour of the block-coordinate sum), each once, in increasing
    even-odd index -- the order of the stored colour maps."""
    for L, b in (((4, 4, 4, 4), (2, 2, 2, 2)), ((8, 8, 8, 8), (4, 4, 4, 4)), ((16, 8, 8, 16), (8, 4, 4, 8)),
                 ((8, 4, 4, 4), (4, 2, 2, 2)), ((12, 12, 12, 12), (6, 6, 6, 6)), ((32, 8, 8, 16), (8, 8, 8, 8))):
        Vh = L[0] * L[1] * L[2] * L[3] // 2
        for p in (0, 1):
            for c in (0, 1):
                hs = []
                for t in range(Vh // 2):
                    h, x = colour_site(L, b, c, t, p)
                    assert (x[0] + x[1] + x[2] + x[3]) % 2 == p
                    assert (x[0] // b[0] + x[1] // b[1] + x[2] // b[2] + x[3] // b[3]) % 2 == c
                    assert h == (x[0] + L[0] * (x[1] + L[1] * (x[2] + L[2] * x[3]))) // 2
                    hs.append(h)
                assert hs == sorted(set(hs)) and len(hs) == Vh // 2
