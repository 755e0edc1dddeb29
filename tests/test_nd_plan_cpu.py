"""Host logic of the nested dissection of P (Sec. 3, Fig. nd; Table cost), no GPU needed.

The planner runs in liblsp.so (lsp_nd_plan_info) and refuses any row pattern whose entries it
cannot assemble exactly once; these tests compare its tree with sizes derived by hand from the
geometry, its flop counts with the formulas of the header, and its refusals.
"""

import pytest

from paper_1607_02560_gb300 import build as B
from paper_1607_02560_gb300 import lsp


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    lsp.lib()


def ring(h, w, n):
    """Points around an h x w box of the n-periodic grid (no wrap-around when h, w < n - 1)."""
    return 2 * (h + w) + 4


def test_n16_leaf8_by_hand():
    # cross: row 0 + column 0 = 31 points; root box 15 x 15 split by its middle column: 15 points,
    # ring = the whole cross (31); halves 15 x 7 split by their middle row: 7 points, ring = 9 + 15
    # + 15 (top and bottom rows coincide: row 16 = row 0); leaves 7 x 7 with a 32-point ring
    info = lsp.nd_plan_info(16, 8)
    assert info["depths"] == [(1, 31, 0), (1, 15, 31), (2, 7, 39), (4, 49, ring(7, 7, 16))]
    assert info["fronts"] == 8 and info["levels"] == 4 and info["max_front"] == 81


def test_n16_leaf4_goes_two_levels_deeper():
    info = lsp.nd_plan_info(16, 4)
    assert info["depths"] == [(1, 31, 0), (1, 15, 31), (2, 7, 39), (4, 7, ring(7, 7, 16)),
                              (8, 3, ring(7, 3, 16)), (16, 9, ring(3, 3, 16))]


@pytest.mark.parametrize("n,leaf,t", [(16, 8, 1), (64, 8, 1), (64, 4, 1), (32, 8, 2), (256, 8, 1)])
def test_every_point_is_eliminated_once_and_flops_follow_the_formulas(n, leaf, t):
    info = lsp.nd_plan_info(n, leaf, t, leaf if t == 2 else 0)
    depths = info["depths"]
    assert sum(c * s for c, s, _ in depths) == n * n
    sweep = sum(c * 2.0 * s * (s + r) ** 2 for c, s, r in depths)
    lu = sum(c * (2.0 / 3.0 * s ** 3 + 2.0 * s * s * r + 2.0 * s * r * r) for c, s, r in depths)
    assert info["flops"] == pytest.approx(sweep, rel=1e-12)
    assert info["flops_lu"] == pytest.approx(lu, rel=1e-12)
    assert info["front_bytes"] == 8 * sum(c * (s + r) ** 2 for c, s, r in depths)
    assert info["solve_bytes"] == 8 * sum(c * ((s + r) * s + s * r) for c, s, r in depths)
    # front counts double with every depth below the root box
    assert [c for c, _, _ in depths] == [1] + [2 ** k for k in range(len(depths) - 1)]
    # the separators are the lines x_a = 0 (mod b): leaves hold (b - 1)^2 points
    assert depths[-1][1] == (leaf - 1) ** 2


def test_cost_grows_like_n_cubed():
    """Table cost, 2D: T_NDsetup = O(N^{3/2} + b^4 N) = O(n^3) at fixed b."""
    f256 = lsp.nd_plan_info(256)["flops_lu"]
    f512 = lsp.nd_plan_info(512)["flops_lu"]
    f1024 = lsp.nd_plan_info(1024)["flops_lu"]
    assert 6.0 < f512 / f256 < 9.0 and 6.0 < f1024 / f512 < 9.0


@pytest.mark.parametrize("args,msg", [
    ((16, 8, 2, 0), "cross the separators"),      # t = 2 everywhere
    ((16, 8, 2, 4), "must equal the nd_leaf"),    # t_j rule of another leaf width
    ((12, 4, 1, 0), "power of two"),
    ((16, 6, 1, 0), "leaf width"),
    ((16, 32, 1, 0), "leaf width"),
    ((2048, 8, 1, 0), "n <= 1024"),
])
def test_plans_that_do_not_fit_are_refused(args, msg):
    with pytest.raises(lsp.LspError, match=msg):
        lsp.nd_plan_info(*args)


def test_3d_n8_leaf4_by_hand():
    # n >= 2b: the torus is opened one axis per depth by the plane pair {x_a = 0} U {x_a = 4}.
    # root: 2 * 8^2 = 128 points; slabs [1, 4) x 8 x 8 (two of them): their points on x_1 = 0, 4,
    # 2 * 3 * 8 = 48, ring = both x_0 planes, 128; bars [1, 4)^2 x 8: their points on x_2 = 0, 4,
    # 2 * 3 * 3 = 18, ring 5 * 5 * 8 - 3 * 3 * 8 = 128; leaves 3^3, ring 5^3 - 27 = 98
    info = lsp.nd_plan_info(8, 4, d=3)
    assert info["depths"] == [(1, 128, 0), (2, 48, 128), (4, 18, 128), (8, 27, 98)]
    # flops from the hand-derived sizes: 2 s (s + r)^2 per front
    sweep = 2.0 * (128 ** 3 + 2 * 48 * 176 ** 2 + 4 * 18 * 146 ** 2 + 8 * 27 * 125 ** 2)
    assert info["flops"] == pytest.approx(sweep, rel=1e-15)


def test_3d_n8_leaf8_keeps_the_three_plane_root():
    # n < 2b: the root is every point with a zero coordinate, 8^3 - 7^3 = 169, and its one child
    # the open cube 7^3, a single leaf whose ring is the whole root
    info = lsp.nd_plan_info(8, 8, d=3)
    assert info["depths"] == [(1, 169, 0), (1, 343, 169)]


@pytest.mark.parametrize("n,leaf", [(8, 4), (16, 8), (32, 4), (16, 16)])
def test_3d_every_point_is_eliminated_once(n, leaf):
    info = lsp.nd_plan_info(n, leaf, d=3)
    depths = info["depths"]
    assert sum(c * s for c, s, _ in depths) == n ** 3
    if n >= 2 * leaf:
        # plane pairs: 2 n^2, then 2 x 2 (n/2 - 1) n, then 4 x 2 (n/2 - 1)^2, then the open
        # cubes (n/2 - 1)^3 split by their middle planes
        h = n // 2 - 1
        assert depths[:3] == [(1, 2 * n * n, 0), (2, 2 * h * n, 2 * n * n),
                              (4, 2 * h * h, (h + 2) ** 2 * n - h * h * n)]
    else:
        assert depths[0] == (1, n ** 3 - (n - 1) ** 3, 0)
    assert depths[-1][1] == (leaf - 1) ** 3
    sweep = sum(c * 2.0 * s * (s + r) ** 2 for c, s, r in depths)
    assert info["flops"] == pytest.approx(sweep, rel=1e-12)


def test_3d_limits_and_multi_t():
    with pytest.raises(lsp.LspError, match="n <= 64"):
        lsp.nd_plan_info(128, 8, d=3)
    with pytest.raises(lsp.LspError, match="cross the separators"):
        lsp.nd_plan_info(16, 8, t=2, nd_leaf=0, d=3)
    # 3D multi-t rows (27 or 125 entries by the leaf-8 t_j rule) fit the leaf-8 dissection
    info = lsp.nd_plan_info(16, 8, t=2, nd_leaf=8, d=3)
    assert sum(c * s for c, s, _ in info["depths"]) == 16 ** 3
