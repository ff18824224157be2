"""The bench's algorithmic-bytes model (bench.phase_bytes, the numerator of
its roofline) against a brute-force count on a HODLR partition (Sec. 2.2,
Fig. 2).  The partition is built here from its definition: leaves
[j L, (j+1) L); a range of leaves [a, b) splits at m = a + (b - a)/2 into the
block rows [m L, b L) x columns [a L, m L) and the two halves.  The test first
checks that the leaf triangles and the blocks tile the lower triangle exactly
once.  It then checks that the model's uncompressed rows, leaf triangles and
factor terms equal the stored elements a sweep at step T must read, counted
one by one."""
import numpy as np
import pytest

import bench


def _partition(nt, L):
    nleaf = (nt + L - 1) // L
    out = {"r0": [], "r1": [], "c0": [], "c1": []}
    stack = [(0, nleaf)]
    while stack:
        a, b = stack.pop()
        if b - a <= 1:
            continue
        m = a + (b - a) // 2
        for key, v in zip(("r0", "r1", "c0", "c1"), (m * L, min(b * L, nt), a * L, m * L)):
            out[key].append(v)
        stack += [(m, b), (a, m)]
    return {key: np.array(v) for key, v in out.items()}


def test_partition_tiles_the_lower_triangle():
    for nt, L in ((1000, 64), (517, 32), (64, 64)):
        blk = _partition(nt, L)
        cover = np.zeros((nt, nt), np.int32)
        for j in range(0, nt, L):
            e = min(j + L, nt)
            cover[j:e, j:e] += np.tril(np.ones((e - j, e - j), np.int32))
        for r0, r1, c0, c1 in zip(blk["r0"], blk["r1"], blk["c0"], blk["c1"]):
            cover[r0:r1, c0:c1] += 1
        assert np.array_equal(cover, np.tril(np.ones((nt, nt), np.int32))), (nt, L)


def test_bytes_model_counts_every_stored_element_once():
    """With the paper's per-step front c = T - k, the model's history H(T)
    equals a one-by-one count: uncompressed rows s >= c (s + 1 elements),
    below c every element either in its leaf triangle or in exactly one block,
    whose factors hold (built rows + columns) x rank elements."""
    nt, L, k, no, r = 1000, 64, 5, 2, 30
    n2 = no * no
    blk = _partition(nt, L)
    rng = np.random.default_rng(3)
    ranks = rng.integers(1, 20, size=(len(blk["r0"]), n2))
    for T, es in ((999, 8), (700, 16), (130, 8)):
        c = T - k
        direct = leaf = inblock = 0
        for s in range(c, T + 1):
            direct += s + 1
        for s in range(c):
            for t in range(s + 1):
                if s // L == t // L:
                    leaf += 1
                else:
                    inblock += 1
        fac = 0
        covered = 0
        for b in range(len(blk["r0"])):
            r0, r1, c0, c1 = blk["r0"][b], blk["r1"][b], blk["c0"][b], blk["c1"][b]
            if r0 < c:
                fac += (min(r1, c) - r0 + (c1 - c0)) * int(ranks[b].sum())
                covered += (min(r1, c) - r0) * (c1 - c0)
        assert covered == inblock                 # the built blocks hold exactly the off-leaf elements
        H = (direct + leaf) * n2 + fac
        row = (T + 1) * n2
        assert bench.history_all_pairs(T, k, L, no, blk, ranks, True) == H
        assert bench.phase_bytes("ret", T, k, no, r, L, es, blk, ranks, True) == H * es + 2 * row * es
        expect_src = H * es + row * es + (T + 1) * r * n2 * 16 + row * 16
        assert bench.phase_bytes("src", T, k, no, r, L, es, blk, ranks, True) == expect_src
        assert bench.phase_flops("les", T, k, no, L, blk, ranks, True) == 8 * no * H
    # dense storage: the whole lower triangle
    assert bench.history_all_pairs(9, 5, 64, 2, None, None, False) == 4 * 55


def test_window_starts_on_a_compression_step():
    for nt, k, L in ((8192, 5, 64), (4096, 5, 64), (2048, 3, 32)):
        T = bench.window_start(nt, k, L, True)
        assert T >= nt // 4 and (T - k) % L == 0 and T - nt // 4 < L
    assert bench.window_start(256, 5, 64, False) == 64


def test_library_partition_matches_the_definition():
    """The partition hkbe_create builds (exported host-only) is the one the
    bench model and the test above use, for every leaf size the library
    accepts, and the library rejects bad sizes."""
    import paper_2604_05319_gb300 as pk
    for nt, L in ((4096, 64), (8192, 64), (1000, 32), (64, 64), (65, 32), (1, 32)):
        lib = pk.hkbe_hodlr_partition(nt, L)
        ref = _partition(nt, L)
        blocks = [sorted(zip(*(p[key].tolist() for key in ("r0", "r1", "c0", "c1")))) for p in (lib, ref)]
        assert blocks[0] == blocks[1], (nt, L)
        assert len(lib["r0"]) == len(ref["r0"]) == max(0, (nt + L - 1) // L - 1)
        assert (lib["level"] >= 0).all() and (np.diff(np.sort(np.unique(lib["level"]))) == 1).all()
    with pytest.raises(pk.HKBEError):
        pk.hkbe_hodlr_partition(0, 64)


def test_code_digest_ignores_comments_only(tmp_path, monkeypatch):
    """A traffic record stays valid across comment edits of the kernel's
    sources and is invalidated by a code edit."""
    csrc = tmp_path / "paper_2604_05319_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_text("// header\nint f(int x) {  /* block\n comment */ return x + 1; }\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    d0 = bench.code_digest(["k.cu"])
    (csrc / "k.cu").write_text("// another header\n\nint f(int x) { return   x + 1; }  // note\n")
    assert bench.code_digest(["k.cu"]) == d0
    (csrc / "k.cu").write_text("int f(int x) { return x + 2; }\n")
    assert bench.code_digest(["k.cu"]) != d0
