// Host planner of the nested dissection of the periodic 2D or 3D grid (Sec. 3, Fig. nd;
// Sec. 4.2; Table cost): the elimination tree, each front's index sets, the child-to-parent
// maps and the list of P's entries assembled into each front. Pure host code; the numeric
// phases are in k_nd.cu.
#include <algorithm>
#include <cstring>

#include "nd.h"

namespace lsp {
namespace {

struct Box {
  int lo[3], len[3];  // points lo[a] .. lo[a] + len[a] - 1 on axis a
  bool cross;         // the 2D (or small 3D) root: every point with a zero coordinate
  bool per[3];        // axis still periodic: lo = 0, len = n, no end on that axis
};

inline int wrapi(int a, int n) {
  a %= n;
  return a < 0 ? a + n : a;
}

// t_j of point x for a t = 2 build with leaf width L (Sec. 4.2): the largest t <= 2 whose
// neighbourhood crosses no line (plane) x_a = 0 (mod L); a point on one counts the full width.
inline int t_point(const int* x, int d, int L) {
  int t = 2;
  for (int a = 0; a < d; ++a) {
    const int rr = x[a] % L;
    const int f = rr == 0 ? L : std::min(rr, L - rr);
    t = std::min(t, f);
  }
  return t;
}

}  // namespace

std::string build_nd_plan(NdPlan& P, int d, int n, int leaf, int t_built, int leaf_t, int mu) {
  P = NdPlan();
  if (d != 2 && d != 3) return "the dissection is built for 2D and 3D grids";
  if (n < 4 || (n & (n - 1))) return "the dissection needs n a power of two >= 4";
  if (leaf < 4 || (leaf & (leaf - 1)) || leaf > n)
    return "the leaf width b must be a power of two with 4 <= b <= n";
  if (t_built == 2 && leaf_t <= 0)
    return "t = 2 rows at every point cross the separators: build with nd_leaf = b";
  if (t_built == 2 && leaf_t != leaf)
    return "the leaf width b must equal the nd_leaf of the multi-t build";
  const int w1 = 2 * t_built + 1;
  if (mu != (d == 2 ? w1 * w1 : w1 * w1 * w1)) return "unexpected row width";
  if (t_built == 2 && n < 8) return "t = 2 rows need n >= 8";
  if (d == 2 && n > kNdMaxN) return "the dissection is built for n <= 1024 in 2D";
  if (d == 3 && n > kNdMaxN3) return "the dissection is built for n <= 64 in 3D";
  P.d = d;
  P.n = n;
  P.leaf = leaf;
  P.mu = mu;
  P.t_built = t_built;
  P.leaf_t = leaf_t;
  const int64_t N = d == 2 ? (int64_t)n * n : (int64_t)n * n * n;
  auto gidx = [&](const int* x) -> int32_t {
    int64_t g = 0;
    for (int a = 0; a < d; ++a) g = g * n + wrapi(x[a], n);
    return (int32_t)g;
  };
  auto coords = [&](int64_t g, int* x) {
    for (int a = d - 1; a >= 0; --a) {
      x[a] = (int)(g % n);
      g /= n;
    }
  };

  // ---- the tree, breadth first: children of front k at depth e are 2k, 2k+1 at depth e+1
  // (the cross has one child). The periodic grid is opened first:
  //  - 2D, or 3D with n < 2b: the root is the cross {some x_a = 0}, its child the open box
  //    [1, n)^d;
  //  - 3D with n >= 2b: one axis per depth, the node's points on the plane pair
  //    {x_a = 0} U {x_a = n/2} (both on multiples of b), children [1, n/2) and [n/2 + 1, n)
  //    on that axis. The separators are the cross's planes and the first middle planes of the
  //    open cube, grouped as 2 n^2, 2 x 2 (n/2 - 1) n, 4 x 2 (n/2 - 1)^2 points instead of
  //    3 n^2 - 3 n + 1, (n - 1)^2, 2 x (n/2 - 1)(n - 1), 4 x (n/2 - 1)^2: the root front
  //    shrinks from 3 n^2 to 2 n^2 points and one depth of large fronts disappears, about a
  //    third of the factorisation's flops at n = 64 (in 2D the two groupings cost the same).
  // An open box is split through the middle plane of its longest side (the first such axis).
  std::vector<std::vector<Box>> boxes;
  const bool pairs = d == 3 && n >= 2 * leaf;
  if (pairs) {
    Box root{};
    for (int a = 0; a < d; ++a) {
      root.lo[a] = 0;
      root.len[a] = n;
      root.per[a] = true;
    }
    boxes.push_back({root});
  } else {
    Box cross{};
    cross.cross = true;
    boxes.push_back({cross});
    Box root{};
    for (int a = 0; a < d; ++a) {
      root.lo[a] = 1;
      root.len[a] = n - 1;
    }
    boxes.push_back({root});
  }
  auto periodic_axis = [&](const Box& b) {
    for (int a = 0; a < d; ++a)
      if (b.per[a]) return a;
    return -1;
  };
  auto is_leaf_box = [&](const Box& b) {
    if (periodic_axis(b) >= 0) return false;
    for (int a = 0; a < d; ++a)
      if (b.len[a] > leaf - 1) return false;
    return true;
  };
  auto split_axis = [&](const Box& b) {
    const int pa = periodic_axis(b);
    if (pa >= 0) return pa;
    int ax = 0;
    for (int a = 1; a < d; ++a)
      if (b.len[a] > b.len[ax]) ax = a;
    return ax;
  };
  while (!is_leaf_box(boxes.back()[0])) {
    std::vector<Box> next;
    next.reserve(boxes.back().size() * 2);
    for (const Box& b : boxes.back()) {
      const int ax = split_axis(b);
      Box c0 = b, c1 = b;
      if (b.per[ax]) {
        c0.per[ax] = c1.per[ax] = false;
        c0.lo[ax] = 1;
        c1.lo[ax] = n / 2 + 1;
        c0.len[ax] = c1.len[ax] = n / 2 - 1;
      } else {
        const int half = (b.len[ax] - 1) / 2;
        c0.len[ax] = half;
        c1.len[ax] = half;
        c1.lo[ax] = b.lo[ax] + half + 1;
      }
      next.push_back(c0);
      next.push_back(c1);
    }
    boxes.push_back(std::move(next));
  }
  const int L = (int)boxes.size();
  P.lv.resize(L);

  std::vector<int32_t> stamp(N, -1);
  int32_t tag = 0;
  // points of the box [lo, lo + len) in lexicographic order, optionally only the plane x_ax = c
  auto for_box = [&](const int* lo, const int* len, auto&& fn) {
    int x[3] = {0, 0, 0};
    const int l2 = d == 3 ? len[2] : 1;
    for (int i = 0; i < len[0]; ++i)
      for (int j = 0; j < len[1]; ++j)
        for (int m = 0; m < l2; ++m) {
          x[0] = lo[0] + i;
          x[1] = lo[1] + j;
          if (d == 3) x[2] = lo[2] + m;
          fn(x);
        }
  };
  auto E_of = [&](const Box& b, bool is_leaf, std::vector<int32_t>& out) {
    if (b.cross) {  // every point with a zero coordinate, lexicographic
      int x[3];
      for (int64_t g = 0; g < N; ++g) {
        coords(g, x);
        bool on = false;
        for (int a = 0; a < d; ++a) on = on || x[a] == 0;
        if (on) out.push_back((int32_t)g);
      }
    } else if (is_leaf) {
      for_box(b.lo, b.len, [&](const int* x) { out.push_back(gidx(x)); });
    } else if (periodic_axis(b) >= 0) {  // the plane pair {x_ax = 0} U {x_ax = n/2}
      const int ax = periodic_axis(b);
      int lo[3] = {b.lo[0], b.lo[1], d == 3 ? b.lo[2] : 0};
      int len[3] = {b.len[0], b.len[1], d == 3 ? b.len[2] : 1};
      len[ax] = 1;
      for (int plane : {0, n / 2}) {
        lo[ax] = plane;
        for_box(lo, len, [&](const int* x) { out.push_back(gidx(x)); });
      }
    } else {
      const int ax = split_axis(b);
      int lo[3] = {b.lo[0], b.lo[1], d == 3 ? b.lo[2] : 0};
      int len[3] = {b.len[0], b.len[1], d == 3 ? b.len[2] : 1};
      lo[ax] = b.lo[ax] + (b.len[ax] - 1) / 2;
      len[ax] = 1;
      for_box(lo, len, [&](const int* x) { out.push_back(gidx(x)); });
    }
  };
  // the ring of a box: the points of its enlarged box [lo - 1, lo + len] (not enlarged along a
  // periodic axis) outside it, wrapped, in lexicographic order of the enlarged box, first copy
  // kept
  auto R_of = [&](const Box& b, std::vector<int32_t>& out) {
    if (b.cross) return;
    ++tag;
    int lo[3] = {0, 0, 0}, len[3] = {1, 1, 1};
    for (int a = 0; a < d; ++a) {
      lo[a] = b.per[a] ? b.lo[a] : b.lo[a] - 1;
      len[a] = b.per[a] ? b.len[a] : b.len[a] + 2;
    }
    for_box(lo, len, [&](const int* x) {
      bool inside = true;
      for (int a = 0; a < d; ++a) inside = inside && x[a] >= b.lo[a] && x[a] < b.lo[a] + b.len[a];
      if (inside) return;
      const int32_t g = gidx(x);
      if (stamp[g] == tag) return;
      stamp[g] = tag;
      out.push_back(g);
    });
  };

  // ---- index sets, depth by depth
  int64_t front_off = 0, perm_off = 0, z_off = 0, u_off = 0, inv_off = 0;
  std::vector<int32_t> e_tmp, r_tmp;
  for (int e = 0; e < L; ++e) {
    NdLevel& lv = P.lv[e];
    const bool is_leaf = e == L - 1;
    lv.count = (int)boxes[e].size();
    lv.nchild = is_leaf ? 0 : (boxes[e][0].cross ? 1 : 2);
    lv.E_off = (int64_t)P.E.size();
    lv.R_off = (int64_t)P.R.size();
    for (int k = 0; k < lv.count; ++k) {
      e_tmp.clear();
      r_tmp.clear();
      E_of(boxes[e][k], is_leaf, e_tmp);
      R_of(boxes[e][k], r_tmp);
      if (k == 0) {
        lv.s = (int)e_tmp.size();
        lv.r = (int)r_tmp.size();
      } else if ((int)e_tmp.size() != lv.s || (int)r_tmp.size() != lv.r) {
        return "internal: fronts of one depth differ in size";
      }
      P.E.insert(P.E.end(), e_tmp.begin(), e_tmp.end());
      P.R.insert(P.R.end(), r_tmp.begin(), r_tmp.end());
    }
    lv.f = lv.s + lv.r;
    if ((double)lv.count * lv.f * lv.f >= 2147483647.0)
      return "the fronts of one depth exceed 2^31 entries (n too large for the dissection)";
    lv.front_off = front_off;
    front_off += (int64_t)lv.count * lv.f * lv.f;
    lv.perm_off = perm_off;
    perm_off += (int64_t)lv.count * lv.s;
    lv.z_off = z_off;
    z_off += (int64_t)lv.count * lv.s;
    lv.u_off = u_off;
    u_off += (int64_t)lv.count * lv.r;
    lv.inv_off = inv_off;
    inv_off += is_leaf ? 0 : (int64_t)lv.count * lv.f * 2;
    const double s = lv.s, r = lv.r, f = lv.f;
    P.flops_sweep += lv.count * 2.0 * s * f * f;
    P.flops_lu += lv.count * (2.0 / 3.0 * s * s * s + 2.0 * s * s * r + 2.0 * s * r * r);
    P.solve_bytes += (int64_t)lv.count * ((int64_t)lv.f * lv.s + (int64_t)lv.s * lv.r) * 8;
    P.max_f = std::max(P.max_f, lv.f);
    P.max_s = std::max(P.max_s, lv.s);
  }
  P.front_doubles = front_off;
  P.perm_ints = perm_off;
  P.z_doubles = z_off;
  P.u_doubles = u_off;
  if ((int64_t)P.E.size() != N) return "internal: the eliminated sets do not cover the grid";
  P.inv.assign(inv_off, -1);

  // ---- assembly lists and child maps
  const int tmax = t_built;
  auto t_of = [&](int32_t g) {
    if (t_built == 1) return 1;
    int x[3];
    coords(g, x);
    return t_point(x, d, leaf_t);
  };
  // offset index in the lexicographic list of [-t_built, t_built]^d (last axis fastest)
  auto a_of = [&](const int* o) {
    int a = 0;
    for (int q = 0; q < d; ++q) a = a * w1 + (o[q] + t_built);
    return a;
  };
  const int nofs = d == 2 ? (2 * tmax + 1) * (2 * tmax + 1)
                          : (2 * tmax + 1) * (2 * tmax + 1) * (2 * tmax + 1);
  std::vector<int32_t> where(N, -1);
  int64_t emitted = 0;
  for (int e = 0; e < L; ++e) {
    NdLevel& lv = P.lv[e];
    lv.asm_off = (int64_t)P.asm_dst.size();
    for (int k = 0; k < lv.count; ++k) {
      const Box& bx = boxes[e][k];
      const int32_t* Ek = P.E.data() + lv.E_off + (int64_t)k * lv.s;
      const int32_t* Rk = P.R.data() + lv.R_off + (int64_t)k * lv.r;
      for (int q = 0; q < lv.s; ++q) where[Ek[q]] = q;
      for (int a = 0; a < lv.r; ++a) where[Rk[a]] = lv.s + a;
      // a point eliminated in this front's subtree before it (inside its box, off E)
      auto descendant = [&](int32_t g) {
        if (where[g] >= 0) return false;
        if (bx.cross) return true;
        int x[3];
        coords(g, x);
        for (int a = 0; a < d; ++a)
          if (x[a] < bx.lo[a] || x[a] >= bx.lo[a] + bx.len[a]) return false;
        return true;
      };
      const int64_t base = (int64_t)k * lv.f * lv.f;
      for (int q = 0; q < lv.s; ++q) {
        const int32_t g = Ek[q];
        int xg[3];
        coords(g, xg);
        const int tg = t_of(g);
        for (int ao = 0; ao < nofs; ++ao) {
          int o[3] = {0, 0, 0}, rem = ao;
          for (int c = d - 1; c >= 0; --c) {
            o[c] = rem % (2 * tmax + 1) - tmax;
            rem /= 2 * tmax + 1;
          }
          bool in_t = true;
          for (int c = 0; c < d; ++c) in_t = in_t && std::abs(o[c]) <= tg;
          int xo[3];
          // row g of P: entry (g, g + o)
          if (in_t) {
            for (int c = 0; c < d; ++c) xo[c] = xg[c] + o[c];
            const int32_t h = gidx(xo);
            if (where[h] >= 0) {
              P.asm_dst.push_back((int32_t)(base + (int64_t)q * lv.f + where[h]));
              P.asm_src.push_back((int32_t)((int64_t)g * mu + a_of(o)));
              ++emitted;
            } else if (!descendant(h)) {
              return "the rows cross a separator of the dissection";
            }
          }
          // column g of P: entry (g - o, g) of a ring row g - o whose pattern holds o
          for (int c = 0; c < d; ++c) xo[c] = xg[c] - o[c];
          const int32_t h = gidx(xo);
          const int th = t_of(h);
          bool in_th = true;
          for (int c = 0; c < d; ++c) in_th = in_th && std::abs(o[c]) <= th;
          if (!in_th) continue;
          if (where[h] >= lv.s) {
            P.asm_dst.push_back((int32_t)(base + (int64_t)where[h] * lv.f + q));
            P.asm_src.push_back((int32_t)((int64_t)h * mu + a_of(o)));
            ++emitted;
          } else if (where[h] < 0 && !descendant(h)) {
            return "the rows cross a separator of the dissection";
          }
        }
      }
      // child ring positions inside this front
      for (int cix = 0; cix < lv.nchild; ++cix) {
        const NdLevel& cl = P.lv[e + 1];
        const int child = lv.nchild == 1 ? k : 2 * k + cix;
        const int32_t* Rc = P.R.data() + cl.R_off + (int64_t)child * cl.r;
        int32_t* inv = P.inv.data() + lv.inv_off + (int64_t)k * lv.f * 2;
        for (int a = 0; a < cl.r; ++a) {
          const int pos = where[Rc[a]];
          if (pos < 0) return "internal: a child's ring leaves its parent's front";
          if (inv[pos * 2 + cix] != -1) return "internal: a child's ring repeats a point";
          inv[pos * 2 + cix] = a;
        }
      }
      for (int q = 0; q < lv.s; ++q) where[Ek[q]] = -1;
      for (int a = 0; a < lv.r; ++a) where[Rk[a]] = -1;
    }
    lv.asm_n = (int64_t)P.asm_dst.size() - lv.asm_off;
  }
  // every structural entry of P assembled exactly once
  int64_t structural = 0;
  for (int64_t g = 0; g < N; ++g) {
    const int tg = t_of((int32_t)g);
    int64_t c = 1;
    for (int a = 0; a < d; ++a) c *= 2 * tg + 1;
    structural += c;
  }
  if (emitted != structural) return "internal: P's entries are not assembled exactly once";
  return "";
}

}  // namespace lsp
