// Host planner of the nested dissection of the periodic 2D grid (Sec. 3, Fig. nd; Sec. 4.2):
// the elimination tree, each front's index sets, the child-to-parent maps and the list of P's
// entries assembled into each front. Pure host code; the numeric phases are in k_nd.cu.
#include <algorithm>
#include <cstring>

#include "nd.h"

namespace lsp {
namespace {

struct Box {
  int i0, j0, h, w;  // rows [i0, i0 + h), columns [j0, j0 + w), inside [1, n)^2
  bool cross;
};

inline int wrapi(int a, int n) {
  a %= n;
  return a < 0 ? a + n : a;
}

// t_j of point (x0, x1) for a t = 2 build with leaf width L (Sec. 4.2): the largest t <= 2
// whose neighbourhood crosses no line x_a = 0 (mod L); a point on a line counts the full width.
inline int t_point(int x0, int x1, int L) {
  int t = 2;
  const int x[2] = {x0, x1};
  for (int a = 0; a < 2; ++a) {
    const int rr = x[a] % L;
    const int f = rr == 0 ? L : std::min(rr, L - rr);
    t = std::min(t, f);
  }
  return t;
}

}  // namespace

std::string build_nd_plan(NdPlan& P, int n, int leaf, int t_built, int leaf_t, int mu) {
  P = NdPlan();
  if (n < 4 || (n & (n - 1))) return "the dissection needs n a power of two >= 4";
  if (leaf < 4 || (leaf & (leaf - 1)) || leaf > n)
    return "the leaf width b must be a power of two with 4 <= b <= n";
  if (t_built == 2 && leaf_t <= 0)
    return "t = 2 rows at every point cross the separators: build with nd_leaf = b";
  if (t_built == 2 && leaf_t != leaf)
    return "the leaf width b must equal the nd_leaf of the multi-t build";
  if ((t_built == 1 && mu != 9) || (t_built == 2 && mu != 25)) return "unexpected row width";
  if (t_built == 2 && n < 8) return "t = 2 rows need n >= 8";
  if (n > kNdMaxN) return "the dissection is built for n <= 1024";
  P.n = n;
  P.leaf = leaf;
  P.mu = mu;
  P.t_built = t_built;
  P.leaf_t = leaf_t;
  const int64_t N = (int64_t)n * n;

  // ---- the tree, breadth first: children of front k at depth d are 2k, 2k+1 at depth d+1
  std::vector<std::vector<Box>> boxes;
  boxes.push_back({Box{0, 0, 0, 0, true}});
  boxes.push_back({Box{1, 1, n - 1, n - 1, false}});
  while (true) {
    const Box& b0 = boxes.back()[0];
    if (b0.h <= leaf - 1 && b0.w <= leaf - 1) break;
    std::vector<Box> next;
    next.reserve(boxes.back().size() * 2);
    for (const Box& b : boxes.back()) {
      if (b.w >= b.h) {
        const int hw = (b.w - 1) / 2;
        next.push_back({b.i0, b.j0, b.h, hw, false});
        next.push_back({b.i0, b.j0 + hw + 1, b.h, hw, false});
      } else {
        const int hh = (b.h - 1) / 2;
        next.push_back({b.i0, b.j0, hh, b.w, false});
        next.push_back({b.i0 + hh + 1, b.j0, hh, b.w, false});
      }
    }
    boxes.push_back(std::move(next));
  }
  const int L = (int)boxes.size();
  P.lv.resize(L);

  std::vector<int32_t> stamp(N, -1);
  int32_t tag = 0;
  auto E_of = [&](const Box& b, bool is_leaf, std::vector<int32_t>& out) {
    if (b.cross) {
      for (int j = 0; j < n; ++j) out.push_back(j);
      for (int i = 1; i < n; ++i) out.push_back(i * n);
    } else if (is_leaf) {
      for (int i = b.i0; i < b.i0 + b.h; ++i)
        for (int j = b.j0; j < b.j0 + b.w; ++j) out.push_back(i * n + j);
    } else if (b.w >= b.h) {
      const int jm = b.j0 + (b.w - 1) / 2;
      for (int i = b.i0; i < b.i0 + b.h; ++i) out.push_back(i * n + jm);
    } else {
      const int im = b.i0 + (b.h - 1) / 2;
      for (int j = b.j0; j < b.j0 + b.w; ++j) out.push_back(im * n + j);
    }
  };
  // the ring of a box in row-major order of its bounding rectangle, wrapped, first copy kept
  auto R_of = [&](const Box& b, std::vector<int32_t>& out) {
    if (b.cross) return;
    ++tag;
    auto add = [&](int i, int j) {
      const int g = wrapi(i, n) * n + wrapi(j, n);
      if (stamp[g] == tag) return;
      stamp[g] = tag;
      out.push_back(g);
    };
    for (int j = b.j0 - 1; j <= b.j0 + b.w; ++j) add(b.i0 - 1, j);
    for (int i = b.i0; i < b.i0 + b.h; ++i) {
      add(i, b.j0 - 1);
      add(i, b.j0 + b.w);
    }
    for (int j = b.j0 - 1; j <= b.j0 + b.w; ++j) add(b.i0 + b.h, j);
  };

  // ---- index sets, level by level
  int64_t front_off = 0, perm_off = 0, z_off = 0, u_off = 0, inv_off = 0;
  std::vector<int32_t> e_tmp, r_tmp;
  for (int d = 0; d < L; ++d) {
    NdLevel& lv = P.lv[d];
    const bool is_leaf = d == L - 1;
    lv.count = (int)boxes[d].size();
    lv.nchild = is_leaf ? 0 : (d == 0 ? 1 : 2);
    lv.E_off = (int64_t)P.E.size();
    lv.R_off = (int64_t)P.R.size();
    for (int k = 0; k < lv.count; ++k) {
      e_tmp.clear();
      r_tmp.clear();
      E_of(boxes[d][k], is_leaf, e_tmp);
      R_of(boxes[d][k], r_tmp);
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
  }
  P.front_doubles = front_off;
  P.perm_ints = perm_off;
  P.z_doubles = z_off;
  P.u_doubles = u_off;
  if ((int64_t)P.E.size() != N) return "internal: the eliminated sets do not cover the grid";
  P.inv.assign(inv_off, -1);

  // ---- assembly lists and child maps
  const int tmax = t_built;
  auto t_of = [&](int g) { return t_built == 1 ? 1 : t_point(g / n, g % n, leaf_t); };
  auto a_of = [&](int o0, int o1) {
    const int w = 2 * t_built + 1;
    return (o0 + t_built) * w + (o1 + t_built);
  };
  std::vector<int32_t> where(N, -1);
  int64_t emitted = 0;
  for (int d = 0; d < L; ++d) {
    NdLevel& lv = P.lv[d];
    lv.asm_off = (int64_t)P.asm_dst.size();
    for (int k = 0; k < lv.count; ++k) {
      const Box& bx = boxes[d][k];
      const int32_t* Ek = P.E.data() + lv.E_off + (int64_t)k * lv.s;
      const int32_t* Rk = P.R.data() + lv.R_off + (int64_t)k * lv.r;
      for (int e = 0; e < lv.s; ++e) where[Ek[e]] = e;
      for (int a = 0; a < lv.r; ++a) where[Rk[a]] = lv.s + a;
      // a point eliminated in this front's subtree before it (inside its box, off E)
      auto descendant = [&](int g) {
        if (bx.cross) return where[g] < 0;
        const int i = g / n, j = g % n;
        return i >= bx.i0 && i < bx.i0 + bx.h && j >= bx.j0 && j < bx.j0 + bx.w &&
               where[g] < 0;
      };
      const int64_t base = (int64_t)k * lv.f * lv.f;
      for (int e = 0; e < lv.s; ++e) {
        const int g = Ek[e];
        const int gi = g / n, gj = g % n;
        // row g of P: entries (g, q) with q in the front
        const int tg = t_of(g);
        for (int o0 = -tg; o0 <= tg; ++o0)
          for (int o1 = -tg; o1 <= tg; ++o1) {
            const int q = wrapi(gi + o0, n) * n + wrapi(gj + o1, n);
            if (where[q] >= 0) {
              P.asm_dst.push_back((int32_t)(base + (int64_t)e * lv.f + where[q]));
              P.asm_src.push_back((int32_t)((int64_t)g * mu + a_of(o0, o1)));
              ++emitted;
            } else if (!descendant(q)) {
              return "the rows cross a separator of the dissection";
            }
          }
        // column g of P: entries (q, g) of ring rows q
        for (int o0 = -tmax; o0 <= tmax; ++o0)
          for (int o1 = -tmax; o1 <= tmax; ++o1) {
            const int q = wrapi(gi - o0, n) * n + wrapi(gj - o1, n);
            const int tq = t_of(q);
            if (std::abs(o0) > tq || std::abs(o1) > tq) continue;
            if (where[q] >= lv.s) {
              P.asm_dst.push_back((int32_t)(base + (int64_t)where[q] * lv.f + e));
              P.asm_src.push_back((int32_t)((int64_t)q * mu + a_of(o0, o1)));
              ++emitted;
            } else if (where[q] < 0 && !descendant(q)) {
              return "the rows cross a separator of the dissection";
            }
          }
      }
      // child ring positions inside this front
      for (int cix = 0; cix < lv.nchild; ++cix) {
        const NdLevel& cl = P.lv[d + 1];
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
      for (int e = 0; e < lv.s; ++e) where[Ek[e]] = -1;
      for (int a = 0; a < lv.r; ++a) where[Rk[a]] = -1;
    }
    lv.asm_n = (int64_t)P.asm_dst.size() - lv.asm_off;
  }
  // every structural entry of P assembled exactly once
  int64_t structural = 0;
  for (int64_t g = 0; g < N; ++g) {
    const int tg = t_of((int)g);
    structural += (2 * tg + 1) * (2 * tg + 1);
  }
  if (emitted != structural) return "internal: P's entries are not assembled exactly once";
  return "";
}

}  // namespace lsp
