// Host planner for the sparse tensor-core stencil sweep.
//
// Sec. 3.1 (Adaptive Layout Morphing): flattening plus horizontal (r1) and vertical (r2)
// duplicate crush turn one stencil step into D = A' B' with A' an m' x k' staircase
// (m' = r1 r2, k' = (k + r1 - 1)(k + r2 - 1)).
// Sec. 3.2 (Structured Sparsity Conversion): Algorithm 1 pairs non-conflicting columns;
// the permutation invariant transformation reorders A' columns (and B' rows) so that every
// group of 4 holds at most 2 nonzeros.
// Sec. 3.3 (Automatic Kernel Generation): the 2:4 metadata and the gather lookup table.
#include "planner.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>

namespace spst {

// ---------------------------------------------------------------------------------------
// Rounding to 16-bit words (RN-even), host side.
// ---------------------------------------------------------------------------------------
static uint32_t f32_bits(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  return u;
}

uint16_t to_half_bits(float x, Word word) {
  if (word == Word::BF16) {
    uint32_t u = f32_bits(x);
    if ((u & 0x7fffffffu) > 0x7f800000u) return 0x7fc0;  // NaN
    uint32_t lsb = (u >> 16) & 1u;
    u += 0x7fffu + lsb;
    return (uint16_t)(u >> 16);
  }
  // FP16: 11-bit significand, exponent range [-14, 15], subnormal step 2^-24.
  double v = (double)x;
  uint16_t sign = std::signbit(v) ? 0x8000 : 0;
  double a = std::fabs(v);
  if (std::isnan(v)) return 0x7e00;
  if (a >= 65520.0) return sign | 0x7c00;  // rounds to infinity
  if (a < std::ldexp(1.0, -14)) {
    double q = std::nearbyint(a * std::ldexp(1.0, 24));  // subnormal units (may reach 1024)
    return sign | (uint16_t)q;                           // 1024 encodes the smallest normal
  }
  int e;
  std::frexp(a, &e);  // a = f * 2^e, f in [0.5, 1)
  e -= 1;             // a = 1.m * 2^e
  double q = std::nearbyint(a * std::ldexp(1.0, 10 - e));  // in [1024, 2048]
  if (q >= 2048.0) {
    q /= 2.0;
    e += 1;
  }
  if (e > 15) return sign | 0x7c00;
  return sign | (uint16_t)((e + 15) << 10) | (uint16_t)((int)q - 1024);
}

float half_bits_to_float(uint16_t h, Word word) {
  if (word == Word::BF16) {
    uint32_t u = (uint32_t)h << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
  }
  int sign = (h >> 15) & 1, e = (h >> 10) & 31, m = h & 1023;
  double v;
  if (e == 0) v = std::ldexp((double)m, -24);
  else if (e == 31) v = m ? NAN : INFINITY;
  else v = std::ldexp(1024.0 + m, e - 25);
  return (float)(sign ? -v : v);
}

// ---------------------------------------------------------------------------------------
// Temporal fusion: the t-fold composition of the offset-indexed kernel (a reading: the
// paper fuses 3 steps "as ConvStencil" without giving the mechanism).
// ---------------------------------------------------------------------------------------
std::vector<double> compose_weights(const std::vector<double>& w, int ndim, int r, int t) {
  std::vector<double> cur = w;
  int rc = r;
  int side0 = 2 * r + 1;
  for (int step = 1; step < t; step++) {
    int rn = rc + r;
    int sc = 2 * rc + 1, sn = 2 * rn + 1;
    int nn = 1;
    for (int i = 0; i < ndim; i++) nn *= sn;
    std::vector<double> nxt((size_t)nn, 0.0);
    int nc = (int)cur.size(), nw = (int)w.size();
    for (int ia = 0; ia < nc; ia++) {
      if (cur[ia] == 0.0) continue;
      int oa[3] = {0, 0, 0}, rem = ia;
      for (int d = ndim - 1; d >= 0; d--) { oa[d] = rem % sc - rc; rem /= sc; }
      for (int ib = 0; ib < nw; ib++) {
        if (w[ib] == 0.0) continue;
        int ob[3] = {0, 0, 0}, rb = ib;
        for (int d = ndim - 1; d >= 0; d--) { ob[d] = rb % side0 - r; rb /= side0; }
        int idx = 0;
        for (int d = 0; d < ndim; d++) idx = idx * sn + (oa[d] + ob[d] + rn);
        nxt[idx] += cur[ia] * w[ib];
      }
    }
    cur.swap(nxt);
    rc = rn;
  }
  return cur;
}

// ---------------------------------------------------------------------------------------
// Algorithm 1: hierarchical two-level matching.
// ---------------------------------------------------------------------------------------
std::vector<std::pair<int, int>> hierarchical_matching(int n, int g, int k) {
  std::vector<std::pair<int, int>> out;
  if (g <= 0 || n % g != 0) return out;
  const int m = n / g;
  const int s1 = std::max(m / 2, k);
  std::vector<char> blk(m, 0);
  std::vector<std::pair<int, int>> M1;
  for (int i = 0; i < m; i++) {
    if (!blk[i] && i + s1 < m && !blk[i + s1]) {
      M1.push_back({i, i + s1});
      blk[i] = blk[i + s1] = 1;
    }
  }
  const int s2 = std::max(g / 2, k);
  std::vector<std::pair<int, int>> M2;
  for (int x = 0; x < m; x++) {
    if (blk[x]) continue;
    std::vector<char> node(g, 0);
    for (int u = 0; u < g; u++) {
      int v = u + s2;
      if (node[u]) continue;
      if (v < g) {
        M2.push_back({x * g + u, x * g + v});
        node[u] = node[v] = 1;
      } else {
        M2.push_back({x * g + u, -1});
        node[u] = 1;
      }
    }
  }
  for (auto& bp : M1)
    for (int t = 0; t < g; t++) out.push_back({bp.first * g + t, bp.second * g + t});
  out.insert(out.end(), M2.begin(), M2.end());
  return out;
}

std::vector<std::pair<int, int>> hierarchical_matching_nd(const std::vector<int>& sizes, int k) {
  if (sizes.size() == 2) return hierarchical_matching(sizes[0] * sizes[1], sizes[1], k);
  std::vector<std::pair<int, int>> out;
  if (sizes.size() < 2) return out;
  const int m = sizes[0];
  int inner = 1;
  for (size_t i = 1; i < sizes.size(); i++) inner *= sizes[i];
  const int s0 = std::max(m / 2, k);
  std::vector<char> matched(m, 0);
  std::vector<std::pair<int, int>> top;
  for (int i = 0; i < m; i++)
    if (!matched[i] && i + s0 < m && !matched[i + s0]) {
      top.push_back({i, i + s0});
      matched[i] = matched[i + s0] = 1;
    }
  for (auto& bp : top)
    for (int t = 0; t < inner; t++) out.push_back({bp.first * inner + t, bp.second * inner + t});
  const std::vector<int> rest(sizes.begin() + 1, sizes.end());
  const auto sub = hierarchical_matching_nd(rest, k);
  for (int x = 0; x < m; x++) {
    if (matched[x]) continue;
    for (auto& pr : sub) out.push_back({x * inner + pr.first, pr.second < 0 ? -1 : x * inner + pr.second});
  }
  return out;
}

// ---------------------------------------------------------------------------------------
// Maximum-cardinality matching in a general graph: Edmonds' blossom algorithm (J. Edmonds,
// "Paths, trees, and flowers", Canadian J. Math. 17, 1965), in its common breadth-first
// textbook formulation with a base array: from each free vertex grow an alternating tree by
// breadth-first search; an edge that closes an odd cycle (a blossom) contracts the cycle
// onto its base (the lowest common base of the edge's ends, found by marking the path from
// one end to the root), whose vertices all become outer vertices of the tree; reaching a
// free vertex gives an augmenting path, which is flipped.  A greedy pass seeds the
// matching.  Returns mate[v] (-1: unmatched).
// ---------------------------------------------------------------------------------------
std::vector<int> max_cardinality_matching(const std::vector<std::vector<int>>& adj) {
  const int n = (int)adj.size();
  std::vector<int> mate(n, -1), parent(n, -1), base(n), queue(n);
  std::vector<char> outer(n, 0), in_blossom(n, 0), seen(n, 0);
  // the first common base of a and b on their paths to the root
  auto common_base = [&](int a, int b) {
    std::fill(seen.begin(), seen.end(), 0);
    for (;;) {
      a = base[a];
      seen[a] = 1;
      if (mate[a] < 0) break;
      a = parent[mate[a]];
    }
    for (;;) {
      b = base[b];
      if (seen[b]) return b;
      b = parent[mate[b]];
    }
  };
  // marks the blossom vertices on the path from v down to base b, re-pointing parents
  auto mark = [&](int v, int b, int child) {
    while (base[v] != b) {
      in_blossom[base[v]] = in_blossom[base[mate[v]]] = 1;
      parent[v] = child;
      child = mate[v];
      v = parent[mate[v]];
    }
  };
  auto augmenting_end = [&](int root) -> int {
    std::fill(outer.begin(), outer.end(), 0);
    std::fill(parent.begin(), parent.end(), -1);
    for (int i = 0; i < n; i++) base[i] = i;
    int head = 0, tail = 0;
    outer[root] = 1;
    queue[tail++] = root;
    while (head < tail) {
      const int v = queue[head++];
      for (int to : adj[v]) {
        if (base[v] == base[to] || mate[v] == to) continue;
        if (to == root || (mate[to] >= 0 && parent[mate[to]] >= 0)) {
          const int b = common_base(v, to);
          std::fill(in_blossom.begin(), in_blossom.end(), 0);
          mark(v, b, to);
          mark(to, b, v);
          for (int i = 0; i < n; i++)
            if (in_blossom[base[i]]) {
              base[i] = b;
              if (!outer[i]) {
                outer[i] = 1;
                queue[tail++] = i;
              }
            }
        } else if (parent[to] < 0) {
          parent[to] = v;
          if (mate[to] < 0) return to;
          outer[mate[to]] = 1;
          queue[tail++] = mate[to];
        }
      }
    }
    return -1;
  };
  for (int v = 0; v < n; v++)
    if (mate[v] < 0)
      for (int to : adj[v])
        if (mate[to] < 0) {
          mate[v] = to;
          mate[to] = v;
          break;
        }
  for (int v = 0; v < n; v++) {
    if (mate[v] >= 0) continue;
    for (int u = augmenting_end(v); u >= 0;) {
      const int pv = parent[u], next = mate[pv];
      mate[u] = pv;
      mate[pv] = u;
      u = next;
    }
  }
  return mate;
}

// ---------------------------------------------------------------------------------------
// Packing matched pairs into K chunks of `slots` (16) pairs so that, within every chunk,
// the first-column offsets and the second-column offsets are distinct mod 16 (see the
// gather's bank rule in build_sweep_tables_2d).  View each pair as an edge between its
// first column's residue (left vertex) and its second column's residue (right vertex) of
// a bipartite multigraph on 16 + 16 vertices; a conflict-free chunk is a matching, so the
// packing is an edge colouring.  Steps: orient each pair (swap its columns) to keep every
// residue's degree small, then colour the edges with max-degree colours by alternating-
// path recolouring (Konig's edge-colouring theorem for bipartite graphs), one chunk per
// colour, and fill each chunk with padding pairs (zero columns) of the unused residues.
// Returns 0, or -1 (order/lut untouched) when no conflict-free packing uses the minimum
// number of chunks (some residue is carried by more than twice that many columns).
// ---------------------------------------------------------------------------------------
int arrange_pairs(const std::vector<std::pair<int, int>>& pairs, const std::vector<std::pair<int, int>>& offs,
                  int slots, std::vector<int>* order_out, std::vector<int32_t>* lut_out) {
  const int n = (int)pairs.size();
  auto res = [](int o) { return ((o % 16) + 16) % 16; };
  // orientation: every residue v needs out(v) <= D and in(v) <= D, where out counts the
  // pairs whose first column has residue v and in those whose second column has.  Choosing
  // which column goes first is a degree-constrained orientation: each pair gives one "out"
  // to one of its two residues, and v must receive between lo(v) = max(0, deg(v) - D) and
  // D of them (deg counts both columns).  Solved as a bipartite b-matching by augmenting
  // paths: first up to lo(v) per residue, then up to D; D starts at the chunk minimum and
  // grows until every pair is placed with every lower bound met.
  std::vector<int> X(n), Y(n);
  for (int i = 0; i < n; i++) {
    X[i] = res(offs[i].first);
    Y[i] = res(offs[i].second);
  }
  std::vector<int> owner(n, -1);  // residue that takes the pair's "out" (its first column)
  const int D = std::max(1, (n + slots - 1) / slots);
  {
    int deg[16] = {0};
    for (int i = 0; i < n; i++) {
      deg[X[i]]++;
      deg[Y[i]]++;
    }
    int load[16] = {0}, cap[16];
    std::fill(owner.begin(), owner.end(), -1);
    // augmenting path search: place pair e on residue v or move another pair off v
    std::function<bool(int, std::vector<char>&)> place = [&](int e, std::vector<char>& seen) -> bool {
      const int cand[2] = {X[e], Y[e]};
      for (int k = 0; k < 2; k++) {
        const int v = cand[k];
        if (k == 1 && Y[e] == X[e]) break;
        if (seen[v]) continue;
        seen[v] = 1;
        if (load[v] < cap[v]) {
          owner[e] = v;
          load[v]++;
          return true;
        }
        for (int f = 0; f < n; f++) {
          if (owner[f] != v || f == e) continue;
          const int other = (X[f] == v) ? Y[f] : X[f];
          if (other == v) continue;
          owner[f] = -1;
          load[v]--;
          if (place(f, seen)) {
            owner[e] = v;
            load[v]++;
            return true;
          }
          owner[f] = v;
          load[v]++;
        }
      }
      return false;
    };
    bool ok = true;
    for (int v = 0; v < 16; v++) ok &= deg[v] <= 2 * D;  // lo(v) <= D is needed
    if (!ok) return -1;  // no conflict-free packing in the minimum number of chunks
    for (int phase = 0; phase < 2 && ok; phase++) {
      for (int v = 0; v < 16; v++) cap[v] = phase == 0 ? std::max(0, deg[v] - D) : D;
      for (int e = 0; e < n; e++) {
        if (owner[e] >= 0) continue;
        std::vector<char> seen(16, 0);
        if (!place(e, seen) && phase == 1) ok = false;
      }
      if (phase == 0)
        for (int v = 0; v < 16; v++) ok &= load[v] >= std::max(0, deg[v] - D);
    }
    if (!ok) return -1;
  }
  std::vector<int> L(n), Rr(n);
  std::vector<char> swp(n, 0);
  for (int i = 0; i < n; i++) {
    swp[i] = owner[i] != X[i];
    L[i] = owner[i];
    Rr[i] = swp[i] ? X[i] : Y[i];
  }
  // colouring: atL[v][c] / atR[v][c] = edge of colour c at vertex v (-1 none)
  std::vector<std::vector<int>> atL(16, std::vector<int>(D, -1)), atR(16, std::vector<int>(D, -1));
  std::vector<int> col(n, -1);
  for (int e = 0; e < n; e++) {
    const int u = L[e], v = Rr[e];
    int a = 0, b = 0;
    while (atL[u][a] >= 0) a++;  // free at u (exists: deg(u) <= D)
    while (atR[v][b] >= 0) b++;  // free at v
    if (atR[v][a] >= 0) {
      // swap colours a and b along the alternating path that starts at v with colour a; it
      // cannot reach u (bipartite parity), so afterwards a is free at both u and v
      std::vector<int> path;
      int side = 1, vert = v, cc = a;  // side 1: right vertex
      while (true) {
        const int f = side ? atR[vert][cc] : atL[vert][cc];
        if (f < 0) break;
        path.push_back(f);
        vert = side ? L[f] : Rr[f];
        side = 1 - side;
        cc = (cc == a) ? b : a;
      }
      for (int f : path) {
        atL[L[f]][col[f]] = -1;
        atR[Rr[f]][col[f]] = -1;
      }
      for (int f : path) {
        col[f] = (col[f] == a) ? b : a;
        atL[L[f]][col[f]] = f;
        atR[Rr[f]][col[f]] = f;
      }
    }
    col[e] = a;
    atL[u][a] = e;
    atR[v][a] = e;
  }
  std::vector<int>& order = *order_out;
  std::vector<int32_t>& lut = *lut_out;
  order.clear();
  lut.clear();
  int repeats = 0;
  for (int c = 0; c < D; c++) {
    int ua[16] = {0}, ub[16] = {0}, cnt = 0;
    for (int e = 0; e < n; e++) {
      if (col[e] != c) continue;
      int a = pairs[e].first, b = pairs[e].second, oa = offs[e].first, ob = offs[e].second;
      if (swp[e]) {
        std::swap(a, b);
        std::swap(oa, ob);
      }
      order.push_back(a);
      order.push_back(b);
      lut.push_back(oa);
      lut.push_back(ob);
      if (ua[res(oa)]++) repeats++;
      if (ub[res(ob)]++) repeats++;
      cnt++;
    }
    // padding pairs: zero columns reading words of the residues the chunk does not use
    for (int s = cnt; s < slots; s++) {
      int ra = 0, rb = 0;
      while (ra < 15 && ua[ra]) ra++;
      while (rb < 15 && ub[rb]) rb++;
      ua[ra]++;
      ub[rb]++;
      order.push_back(-1);
      order.push_back(-1);
      lut.push_back(ra);
      lut.push_back(rb);
    }
  }
  return repeats;
}

// Packs pairs into chunks of `slots` pairs with as few residue repeats as a local search
// finds, for when no conflict-free packing in the minimum number of chunks exists.  A repeat
// is a second column offset of the same residue mod 16 on the same side (first or second
// columns) of one chunk: it costs the gather one extra shared-memory wavefront.  Offsets of
// -1 mark zero columns, which read any word (their weights are zero) and so take a residue
// the chunk's side does not use.  Moves: exchange two pairs (or a pair and an empty slot)
// between chunks, each pair in either orientation, accepted when the repeat count does not
// grow; a fixed-seed generator keeps the result deterministic.  Returns the repeat count.
int pack_pairs_min_repeats(const std::vector<std::pair<int, int>>& pairs, const std::vector<std::pair<int, int>>& offs,
                           int slots, std::vector<int>* order_out, std::vector<int32_t>* lut_out) {
  const int n = (int)pairs.size();
  const int nch = std::max(1, (n + slots - 1) / slots);
  const int nslot = nch * slots;
  auto res = [](int o) { return o < 0 ? -1 : ((o % 16) + 16) % 16; };
  // slot s holds item it[s] (-1 empty) with flip fl[s]
  std::vector<int> it(nslot, -1);
  std::vector<char> fl(nslot, 0);
  for (int i = 0; i < n; i++) it[i] = i;
  auto rA = [&](int s) { return it[s] < 0 ? -1 : res(fl[s] ? offs[it[s]].second : offs[it[s]].first); };
  auto rB = [&](int s) { return it[s] < 0 ? -1 : res(fl[s] ? offs[it[s]].first : offs[it[s]].second); };
  std::vector<int> cA(nch * 16, 0), cB(nch * 16, 0);
  for (int s = 0; s < nslot; s++) {
    const int c = s / slots, a = rA(s), b = rB(s);
    if (a >= 0) cA[c * 16 + a]++;
    if (b >= 0) cB[c * 16 + b]++;
  }
  int total = 0;
  for (int i = 0; i < nch * 16; i++) total += std::max(0, cA[i] - 1) + std::max(0, cB[i] - 1);
  // repeat-count change when residue r leaves (d = -1) or joins (d = +1) counter x
  auto dlt = [](int x, int d) { return d > 0 ? (x >= 1 ? 1 : 0) : (x >= 2 ? -1 : 0); };
  uint64_t st = 0x9E3779B97F4A7C15ull;
  auto rnd = [&](uint64_t m) {
    st ^= st << 13;
    st ^= st >> 7;
    st ^= st << 17;
    return (int)(st % m);
  };
  // a lower bound: a residue carried by more columns than the chunk sides offer repeats
  int bound = 0;
  {
    int deg[16] = {0};
    for (int i = 0; i < n; i++) {
      if (res(offs[i].first) >= 0) deg[res(offs[i].first)]++;
      if (res(offs[i].second) >= 0) deg[res(offs[i].second)]++;
    }
    for (int v = 0; v < 16; v++) bound += std::max(0, deg[v] - 2 * nch);
  }
  std::vector<int> best_it = it;
  std::vector<char> best_fl = fl;
  int best = total;
  const long iters = 300000;
  for (long k = 0; k < iters && best > bound; k++) {
    const int s1 = rnd(nslot), s2 = rnd(nslot);
    const int c1 = s1 / slots, c2 = s2 / slots;
    if (c1 == c2 || (it[s1] < 0 && it[s2] < 0)) continue;
    const int f1 = rnd(2), f2 = rnd(2);  // new orientations of the items moving into c2 / c1
    auto resA = [&](int s, int f) { return it[s] < 0 ? -1 : res(f ? offs[it[s]].second : offs[it[s]].first); };
    auto resB = [&](int s, int f) { return it[s] < 0 ? -1 : res(f ? offs[it[s]].first : offs[it[s]].second); };
    const int a1 = rA(s1), b1 = rB(s1), a2 = rA(s2), b2 = rB(s2);
    const int na1 = resA(s1, f1), nb1 = resB(s1, f1), na2 = resA(s2, f2), nb2 = resB(s2, f2);
    // item of s1 leaves c1 and joins c2; item of s2 leaves c2 and joins c1
    int d = 0;
    if (a1 >= 0) { d += dlt(cA[c1 * 16 + a1], -1); cA[c1 * 16 + a1]--; }
    if (b1 >= 0) { d += dlt(cB[c1 * 16 + b1], -1); cB[c1 * 16 + b1]--; }
    if (a2 >= 0) { d += dlt(cA[c2 * 16 + a2], -1); cA[c2 * 16 + a2]--; }
    if (b2 >= 0) { d += dlt(cB[c2 * 16 + b2], -1); cB[c2 * 16 + b2]--; }
    if (na1 >= 0) { d += dlt(cA[c2 * 16 + na1], +1); cA[c2 * 16 + na1]++; }
    if (nb1 >= 0) { d += dlt(cB[c2 * 16 + nb1], +1); cB[c2 * 16 + nb1]++; }
    if (na2 >= 0) { d += dlt(cA[c1 * 16 + na2], +1); cA[c1 * 16 + na2]++; }
    if (nb2 >= 0) { d += dlt(cB[c1 * 16 + nb2], +1); cB[c1 * 16 + nb2]++; }
    // annealing: a move that adds one repeat is taken with a probability falling from 1/8
    // to 0 over the run
    const bool take = d <= 0 || (d == 1 && (uint64_t)rnd(1u << 20) < (uint64_t)((1u << 17) * (iters - k) / iters));
    if (take) {
      std::swap(it[s1], it[s2]);
      fl[s2] = (char)f1;
      fl[s1] = (char)f2;
      total += d;
      if (total < best) {
        best = total;
        best_it = it;
        best_fl = fl;
      }
    } else {  // undo
      if (na1 >= 0) cA[c2 * 16 + na1]--;
      if (nb1 >= 0) cB[c2 * 16 + nb1]--;
      if (na2 >= 0) cA[c1 * 16 + na2]--;
      if (nb2 >= 0) cB[c1 * 16 + nb2]--;
      if (a1 >= 0) cA[c1 * 16 + a1]++;
      if (b1 >= 0) cB[c1 * 16 + b1]++;
      if (a2 >= 0) cA[c2 * 16 + a2]++;
      if (b2 >= 0) cB[c2 * 16 + b2]++;
    }
  }
  it = best_it;
  fl = best_fl;
  total = best;
  std::vector<int>& order = *order_out;
  std::vector<int32_t>& lut = *lut_out;
  order.clear();
  lut.clear();
  for (int c = 0; c < nch; c++) {
    int ua[16] = {0}, ub[16] = {0};
    for (int j = 0; j < slots; j++) {
      const int s = c * slots + j;
      if (rA(s) >= 0) ua[rA(s)]++;
      if (rB(s) >= 0) ub[rB(s)]++;
    }
    for (int j = 0; j < slots; j++) {
      const int s = c * slots + j;
      int ca = -1, cb = -1, oa = -1, ob = -1;
      if (it[s] >= 0) {
        const int e = it[s];
        ca = fl[s] ? pairs[e].second : pairs[e].first;
        cb = fl[s] ? pairs[e].first : pairs[e].second;
        oa = fl[s] ? offs[e].second : offs[e].first;
        ob = fl[s] ? offs[e].first : offs[e].second;
      }
      // zero columns read row 0 of the patch window at a residue this side does not use
      if (oa < 0) {
        int r = 0;
        while (r < 15 && ua[r]) r++;
        ua[r]++;
        oa = r;
      }
      if (ob < 0) {
        int r = 0;
        while (r < 15 && ub[r]) r++;
        ub[r]++;
        ob = r;
      }
      order.push_back(ca);
      order.push_back(cb);
      lut.push_back(oa);
      lut.push_back(ob);
    }
  }
  return total;
}

// ---------------------------------------------------------------------------------------
// 2D sweep tables.
// ---------------------------------------------------------------------------------------
std::string build_sweep_tables_2d(const std::vector<double>& wfused, int R, const PlanGeometry& geo, Word word,
                                  int max_pieces, bool drop_zero_pairs, SweepTables* out, Pairing pairing) {
  SweepTables& T = *out;
  T = SweepTables();
  const bool d3 = geo.ndim == 3, d1 = geo.ndim == 1;
  T.ndim = geo.ndim;
  T.R = R;
  T.kt = 2 * R + 1;
  const int kt = T.kt;
  // 1D: one staircase block (r2 = r3 = 1), so the 2D formulas below hold with mb = 1
  const int r1 = d1 ? Tile1D::R1 : (d3 ? Tile3D::R1 : geo.r1);
  const int r2 = d1 ? 1 : (d3 ? Tile3D::R2 : geo.r2), r3 = d3 ? Tile3D::R3 : 1;
  const int M = d1 ? Tile1D::M : (d3 ? Tile3D::M : Tile2D::M);
  if (!d1 && !d3 && (r1 * r2 != Tile2D::M || (r1 != 16 && r1 != 8))) return "2D patches are 16 x 8 or 8 x 16";
  T.r1 = r1;
  T.r2 = r2;
  T.r3 = r3;
  T.g = kt + r1 - 1;
  T.mb = d1 ? 1 : kt + r2 - 1;
  T.mz = d3 ? kt + r3 - 1 : 1;
  T.kprime = T.g * T.mb * T.mz;
  if ((int)wfused.size() != (d3 ? kt * kt * kt : (d1 ? kt : kt * kt))) return "fused weight cube has the wrong size";
  T.wfused = wfused;
  T.wfused32.resize(wfused.size());
  double S = 0.0;
  for (size_t i = 0; i < wfused.size(); i++) {
    T.wfused32[i] = (float)wfused[i];
    S += wfused[i];
  }
  T.S = S;
  T.S_hi = (float)S;
  T.S_lo = (float)(S - (double)T.S_hi);

  // Staircase A' (Sec. 3.1): row rho = s*r1 + tau, column kappa = u*g + c,
  // A'[rho][kappa] = w[u - s][c - tau] when both differences lie in [0, kt).  3D (a third
  // crush along z, nested one level deeper): row rho = (q*r2 + s)*r1 + tau, column
  // kappa = (v*mb + u)*g + c, A'[rho][kappa] = w[v - q][u - s][c - tau].
  const int g = T.g, mb = T.mb, kp = T.kprime;
  auto aval = [&](int rho, int kappa) -> float {
    const int tau = rho % r1, s = (rho / r1) % r2, q = rho / (r1 * r2);
    const int c = kappa % g, u = (kappa / g) % mb, v = kappa / (g * mb);
    const int dz = v - q, dy = u - s, dx = c - tau;
    if (dz < 0 || dz >= (d3 ? kt : 1) || dy < 0 || dy >= kt || dx < 0 || dx >= kt) return 0.f;
    return T.wfused32[(dz * kt + dy) * kt + dx];
  };
  std::vector<char> colnz(kp, 0);
  for (int kap = 0; kap < kp; kap++)
    for (int rho = 0; rho < M && !colnz[kap]; rho++)
      if (aval(rho, kap) != 0.f) colnz[kap] = 1;

  // Structured sparsity conversion (Sec. 3.2).
  auto pairs = d3 ? hierarchical_matching_nd({T.mz, mb, g}, kt) : hierarchical_matching(kp, g, kt);
  std::vector<std::pair<int, int>> kept;
  for (auto& pr : pairs) {
    bool a_nz = colnz[pr.first];
    bool b_nz = pr.second >= 0 && colnz[pr.second];
    if (pr.second < 0) T.zero_cols++;
    if (drop_zero_pairs && !a_nz && !b_nz) {
      T.dropped_pairs++;
      continue;
    }
    kept.push_back(pr);
  }
  // A support smaller than the box (stars, custom masks) leaves A' columns that are zero, and
  // Algorithm 1's block pairing, built for the full staircase, may then pad more than needed.
  // Problem 1 on the actual support is a maximum matching in the graph of nonzero columns
  // whose row supports are disjoint (such a pair holds at most one nonzero per row); it is
  // taken when it needs fewer 32-row K chunks.
  std::vector<int> nzcols;
  for (int kap = 0; kap < kp; kap++)
    if (colnz[kap]) nzcols.push_back(kap);
  if (drop_zero_pairs && (int)nzcols.size() < kp && pairing != Pairing::Algorithm1) {
    const int n = (int)nzcols.size();
    std::vector<std::vector<uint64_t>> rows(n, std::vector<uint64_t>((size_t)(M + 63) / 64, 0));
    for (int i = 0; i < n; i++)
      for (int rho = 0; rho < M; rho++)
        if (aval(rho, nzcols[i]) != 0.f) rows[i][rho / 64] |= 1ull << (rho % 64);
    std::vector<std::vector<int>> adj(n);
    for (int i = 0; i < n; i++)
      for (int j = i + 1; j < n; j++) {
        bool disjoint = true;
        for (size_t wd = 0; wd < rows[i].size() && disjoint; wd++) disjoint = (rows[i][wd] & rows[j][wd]) == 0;
        if (disjoint) {
          adj[i].push_back(j);
          adj[j].push_back(i);
        }
      }
    const std::vector<int> mate = max_cardinality_matching(adj);
    std::vector<std::pair<int, int>> mpairs;
    int unmatched = 0;
    for (int i = 0; i < n; i++) {
      if (mate[i] < 0) {
        mpairs.push_back({nzcols[i], -1});
        unmatched++;
      } else if (i < mate[i]) {
        mpairs.push_back({nzcols[i], nzcols[mate[i]]});
      }
    }
    const int chunk_pairs = Tile2D::KCHUNK / 2;
    if (pairing == Pairing::Matching ||
        (mpairs.size() + chunk_pairs - 1) / chunk_pairs < (kept.size() + chunk_pairs - 1) / chunk_pairs) {
      kept = std::move(mpairs);
      T.zero_cols = unmatched;
      T.dropped_pairs = 0;
      T.pairing = 1;
    }
  }
  // Lookup-table offsets (Sec. 3.3): tile word of column (u, c) relative to the patch base
  // (py*R2*P + px*R1).  The tile starts G cells before the tile's first output, the patch
  // window R cells before the patch's first output.  A zero column reads its pair partner
  // (any finite value works: its weights are zero).
  // 3D: a tile plane holds box_h rows of P words, and the patch window starts R planes
  // before the patch's first output plane as well.
  auto off = [&](int col) {
    const int c = col % g, u = (col / g) % mb, v = col / (g * mb);
    const int plane = geo.box_h * geo.P;
    if (d1) return c + geo.G - R;  // the line is contiguous in the tile
    return (d3 ? (v + geo.G - R) * plane : 0) + (u + geo.G - R) * geo.P + (c + geo.G - R);
  };
  std::vector<std::pair<int, int>> offs;
  for (auto& pr : kept) offs.push_back({off(pr.first), pr.second >= 0 ? off(pr.second) : off(pr.first)});
  std::vector<std::pair<int, int>> offs_free;  // zero partners marked -1: they may read any word
  for (auto& pr : kept) offs_free.push_back({off(pr.first), pr.second >= 0 ? off(pr.second) : -1});
  // Each matched pair holds at most one nonzero per row (its columns are >= kt apart, or one
  // is a zero column), so any two pairs form a valid group of four: the pairs may be
  // reordered and each pair's two columns swapped without breaking 2:4.  Use that freedom
  // for the gather: chunk slot p (pair p of a 32-row K chunk) is read by lane p of both
  // half-warps, whose patches are 16 words apart, so the loads are free of bank conflicts
  // when the chunk's 16 first-column offsets, and its 16 second-column offsets, are distinct
  // mod 16.  arrange_pairs packs the pairs into chunks that way (padding pairs fill the
  // gaps with offsets of the missing residues).
  std::vector<int> order;
  std::vector<int32_t> lut;
  if (arrange_pairs(kept, offs, Tile2D::KCHUNK / 2, &order, &lut) < 0) {
    // no conflict-free packing in the minimum number of chunks: the fewest repeats a local
    // search finds, starting from Algorithm 1's order
    T.bank_conflicts = pack_pairs_min_repeats(kept, offs_free, Tile2D::KCHUNK / 2, &order, &lut);
  }
  T.order = order;
  const int kpad = (int)order.size();
  T.kpad = kpad;
  const int half = kpad / 2;

  // Weight pieces: w * 2^s = p0 + p1 + p2, each RN-even in the 16-bit word.  FP16 scales
  // the weights so that the largest is in [2^10, 2^11): the third piece of every weight within
  // a factor 2^10 of the largest then stays a normal FP16 number, and three pieces (3 x 11
  // significand bits) hold it exactly; BF16 has FP32's exponent range, uses s = 0, and three
  // BF16 pieces hold an FP32 weight exactly (3 x 8 significand bits).
  if (max_pieces < 1 || max_pieces > 3) return "bad piece count";
  double wmax = 0.0;
  for (float v : T.wfused32) wmax = std::max(wmax, (double)std::fabs(v));
  int s = 0;
  if (word == Word::FP16 && wmax > 0.0) {
    int e;
    std::frexp(wmax, &e);  // wmax = f * 2^e, f in [0.5, 1)
    s = 11 - e;            // largest scaled weight in [2^10, 2^11)
  }
  T.wscale_log2 = s;
  // Compression with 2:4 metadata (Sec. 3.3, Metadata; Sec. 2.1 for sub-2:4 groups).
  for (int pc = 0; pc < 3; pc++) T.a_val[pc].assign((size_t)M * half, 0.f);
  T.a_idx.assign((size_t)M * half, 0);
  bool piece_used[3] = {false, false, false};
  for (int rho = 0; rho < M; rho++) {
    for (int q = 0; q < kpad / 4; q++) {
      int pos[4], nnz = 0;
      float val[4];
      for (int e = 0; e < 4; e++) {
        int col = order[4 * q + e];
        float v = col >= 0 ? aval(rho, col) : 0.f;
        if (v != 0.f) {
          if (nnz >= 2) return "permuted staircase violates 2:4 (row " + std::to_string(rho) + ")";
          pos[nnz] = e;
          val[nnz] = v;
          nnz++;
        }
      }
      // fill sub-2:4 groups with the lowest unused positions (their values are zero)
      for (int e = 0; nnz < 2 && e < 4; e++) {
        bool used = false;
        for (int j = 0; j < nnz; j++) used |= (pos[j] == e);
        if (!used) {
          pos[nnz] = e;
          val[nnz] = 0.f;
          nnz++;
        }
      }
      if (pos[0] > pos[1]) {
        std::swap(pos[0], pos[1]);
        std::swap(val[0], val[1]);
      }
      for (int j = 0; j < 2; j++) {
        size_t at = (size_t)rho * half + 2 * q + j;
        float rem = std::ldexp(val[j], s);  // exact (power-of-two scale)
        for (int pc = 0; pc < max_pieces; pc++) {
          float hv = half_bits_to_float(to_half_bits(rem, word), word);
          T.a_val[pc][at] = hv;
          if (hv != 0.f) piece_used[pc] = true;
          rem -= hv;  // exact: the residual of a round-to-nearest is representable
        }
        T.a_idx[at] = (uint8_t)pos[j];
      }
    }
  }
  T.a_pieces = 1;
  for (int pc = 1; pc < max_pieces; pc++)
    if (piece_used[pc]) T.a_pieces = pc + 1;
  // TMEM image of A'' (lane = row; column j holds compressed elements 2j (low) and 2j+1).
  const int pieces = T.a_pieces;
  const int wcols = kpad / 4;
  T.a_words.assign((size_t)pieces * M * wcols, 0u);
  for (int p = 0; p < pieces; p++)
    for (int rho = 0; rho < M; rho++)
      for (int j = 0; j < wcols; j++) {
        const std::vector<float>& src = T.a_val[p];
        uint32_t lo = to_half_bits(src[(size_t)rho * half + 2 * j], word);
        uint32_t hi = to_half_bits(src[(size_t)rho * half + 2 * j + 1], word);
        T.a_words[((size_t)p * M + rho) * wcols + j] = lo | (hi << 16);
      }
  // TMEM image of the metadata: one column per 32-wide K chunk.  Row rho's chunk word has
  // nibble (idx0 | idx1 << 2) for group q at bits 4q.  In each block of 16 lanes, row rr < 8
  // keeps its groups 0-3 in lane rr bits [0,16) and groups 4-7 in lane rr+8 bits [0,16);
  // row rr >= 8 keeps groups 0-3 in lane rr-8 bits [16,32) and groups 4-7 in lane rr
  // bits [16,32).  (Layout measured on sm_103a for kind::f16, M = 128, selector 0.)
  const int nch = kpad / Tile2D::KCHUNK;
  T.meta_words.assign((size_t)M * nch, 0u);
  for (int kc = 0; kc < nch; kc++) {
    for (int rho = 0; rho < M; rho++) {
      uint32_t wrow = 0;
      for (int q = 0; q < 8; q++) {
        size_t at = (size_t)rho * half + kc * 16 + 2 * q;
        wrow |= (uint32_t)(T.a_idx[at] | (T.a_idx[at + 1] << 2)) << (4 * q);
      }
      uint32_t lo16 = wrow & 0xffffu, hi16 = wrow >> 16;
      int base = rho & ~15, rr = rho & 15;
      if (rr < 8) {
        T.meta_words[(size_t)(base + rr) * nch + kc] |= lo16;
        T.meta_words[(size_t)(base + rr + 8) * nch + kc] |= hi16;
      } else {
        T.meta_words[(size_t)(base + rr - 8) * nch + kc] |= lo16 << 16;
        T.meta_words[(size_t)(base + rr) * nch + kc] |= hi16 << 16;
      }
    }
  }
  T.lut = lut;
  (void)mb;
  return "";
}

std::vector<uint32_t> dense_a_words(const SweepTables& T, Word word) {
  const int M = 128, half = T.kpad / 2, dcols = T.kpad / 2;
  std::vector<uint32_t> out((size_t)T.a_pieces * M * dcols, 0u);
  std::vector<float> row((size_t)T.kpad);
  for (int p = 0; p < T.a_pieces; p++)
    for (int rho = 0; rho < M; rho++) {
      std::fill(row.begin(), row.end(), 0.f);
      for (int j = 0; j < half; j++) {
        const size_t at = (size_t)rho * half + j;
        row[(size_t)(j / 2) * 4 + T.a_idx[at]] = T.a_val[p][at];
      }
      for (int c = 0; c < dcols; c++)
        out[((size_t)p * M + rho) * dcols + c] =
            (uint32_t)to_half_bits(row[2 * c], word) | ((uint32_t)to_half_bits(row[2 * c + 1], word) << 16);
    }
  return out;
}

// ---------------------------------------------------------------------------------------
// Cost model of Sec. 3.3: T = max(T_compute, T_memory), with
//   T_compute = N_MMA * CPI / (f N_tcu)  (here: executed sparse MMA flops / tensor rate),
//   T_memory  = max((data_R + data_W) / bw_G, (data_transW + data_transR) / bw_S),
//   data_transR = data_transW = k' (m'/2 + n') elements (reading: m means m').
// ---------------------------------------------------------------------------------------
double layout_cost_seconds(int kt, int r1, int r2, int64_t H, int64_t W, int kpad, double tensor_flops,
                           double hbm_bytes_per_s, double smem_bytes_per_s) {
  const double mprime = (double)r1 * r2;
  const double kprime = (double)(kt + r1 - 1) * (kt + r2 - 1);
  const double nprime = (double)H * (double)W / mprime;
  const double n_mma = std::ceil(mprime / 128.0) * std::ceil((double)kpad / 32.0) * std::ceil(nprime / 128.0);
  const double t_compute = n_mma * 2.0 * 128.0 * 128.0 * 32.0 / tensor_flops;
  const double data_rw = 8.0 * (double)H * (double)W;
  const double trans = kprime * (mprime / 2.0 + nprime) * 2.0;
  const double t_memory = std::max(data_rw / hbm_bytes_per_s, 2.0 * trans / smem_bytes_per_s);
  return std::max(t_compute, t_memory);
}

}  // namespace spst
