// Host-side graph layer: vertex graphs without lepton loops, their mirror
// images, gauge classes, UV-divergent subgraphs, forests, the UV degree,
// I-closures and the Deg set function (Sec. 2 and Sec. 3 of arXiv:1905.08007).
//
// Conventions (a definition both sides of the project state independently):
//   * photon vertices 0..2n-1 along the electron flow, the external vertex X
//     after the first e of them (1 <= e <= 2n-1);
//   * positions 0..2n on the electron line, X at position e;
//   * electron line i joins positions i and i+1 (i = 0..2n-1);
//   * photons sorted by first vertex; line index: electrons 0..2n-1, then
//     photons 2n..3n-1.
#pragma once
#include <algorithm>
#include <array>
#include <cstdint>
#include <functional>
#include <map>
#include <stdexcept>
#include <string>
#include <vector>

namespace qed {

struct Graph {
  int n = 0;                                   // loops = photons
  std::vector<std::pair<int, int>> ph;         // photon endpoints (s < t), sorted
  int e = 0;                                   // X after e photon vertices

  int n_lines() const { return 3 * n; }
  int n_elec() const { return 2 * n; }
  int pos(int v) const { return v < e ? v : v + 1; }
  std::pair<int, int> ph_pos(int a) const { return {pos(ph[a].first), pos(ph[a].second)}; }
  // electron lines carrying photon a's loop momentum
  std::pair<int, int> span(int a) const { auto p = ph_pos(a); return {p.first, p.second - 1}; }
  std::pair<int, int> line_ends(int l) const {
    if (l < n_elec()) return {l, l + 1};
    return ph_pos(l - n_elec());
  }
  // photon attached at position p (p != e)
  int photon_at(int p) const {
    int v = p < e ? p : p - 1;
    for (int a = 0; a < n; ++a) if (ph[a].first == v || ph[a].second == v) return a;
    throw std::logic_error("no photon at position");
  }
  std::vector<int> key() const {
    std::vector<int> k;
    for (auto &p : ph) { k.push_back(p.first); k.push_back(p.second); }
    k.push_back(e);
    return k;
  }
  Graph mirror() const {
    Graph g; g.n = n; g.e = 2 * n - e;
    int m = 2 * n - 1;
    for (auto &p : ph) g.ph.push_back({std::min(m - p.first, m - p.second), std::max(m - p.first, m - p.second)});
    std::sort(g.ph.begin(), g.ph.end());
    return g;
  }
  bool self_mirror() const { return mirror().key() == key(); }
  std::array<int, 3> gauge_class() const {
    int k = 0, l = 0, r = 0;
    for (auto &p : ph) {
      if (p.second < e) ++l; else if (p.first >= e) ++r; else ++k;
    }
    return {k, std::max(l, r), std::min(l, r)};
  }
  std::string name() const {
    std::string s = "n" + std::to_string(n) + "_e" + std::to_string(e);
    for (auto &p : ph) s += "_" + std::to_string(p.first) + std::to_string(p.second);
    return s;
  }
};

inline bool closed_under(const Graph &g, int lo, int hi) {   // vertices lo..hi-1
  for (auto &p : g.ph) {
    bool a = p.first >= lo && p.first < hi, b = p.second >= lo && p.second < hi;
    if (a != b) return false;
  }
  return true;
}

// Admissible: no self-energy on an external leg, one-particle irreducible.
inline bool admissible(const Graph &g) {
  for (int k = 1; k <= g.e; ++k) if (closed_under(g, 0, k)) return false;
  for (int k = g.e; k < 2 * g.n; ++k) if (closed_under(g, k, 2 * g.n)) return false;
  return true;
}

inline void matchings_rec(std::vector<int> &rest, std::vector<std::pair<int, int>> &cur,
                          std::vector<std::vector<std::pair<int, int>>> &out) {
  if (rest.empty()) { auto c = cur; std::sort(c.begin(), c.end()); out.push_back(c); return; }
  int a = rest[0];
  for (size_t i = 1; i < rest.size(); ++i) {
    int b = rest[i];
    std::vector<int> r2;
    for (size_t j = 1; j < rest.size(); ++j) if (j != i) r2.push_back(rest[j]);
    cur.push_back({a, b});
    matchings_rec(r2, cur, out);
    cur.pop_back();
  }
}

// All graphs of order n, both orientations, in a fixed order
// (pairings in lexicographic order, then e ascending).
inline std::vector<Graph> enumerate_graphs(int n) {
  std::vector<int> vs(2 * n);
  for (int i = 0; i < 2 * n; ++i) vs[i] = i;
  std::vector<std::vector<std::pair<int, int>>> ms;
  std::vector<std::pair<int, int>> cur;
  matchings_rec(vs, cur, ms);
  std::sort(ms.begin(), ms.end());
  std::vector<Graph> out;
  for (auto &m : ms)
    for (int e = 1; e < 2 * n; ++e) {
      Graph g; g.n = n; g.ph = m; g.e = e;
      if (admissible(g)) out.push_back(g);
    }
  return out;
}

// ---------------------------------------------------------------------------
// UV degree, I-closure, Deg
// ---------------------------------------------------------------------------
inline int omega(const Graph &g, uint32_t s) {
  int N = g.n_lines();
  std::vector<int> parent(2 * g.n + 1);
  std::vector<char> used(2 * g.n + 1, 0);
  for (int i = 0; i <= 2 * g.n; ++i) parent[i] = i;
  std::function<int(int)> find = [&](int x) { while (parent[x] != x) x = parent[x] = parent[parent[x]]; return x; };
  int nl = 0, nph = 0, nv = 0, comps = 0;
  for (int l = 0; l < N; ++l) if (s >> l & 1) {
    ++nl; if (l >= g.n_elec()) ++nph;
    auto ends = g.line_ends(l);
    for (int v : {ends.first, ends.second}) if (!used[v]) { used[v] = 1; ++nv; ++comps; }
  }
  for (int l = 0; l < N; ++l) if (s >> l & 1) {
    auto ends = g.line_ends(l);
    int a = find(ends.first), b = find(ends.second);
    if (a != b) { parent[a] = b; --comps; }
  }
  int loops = nl - nv + comps;
  return 4 * loops - 2 * nph - (nl - nph);
}

inline uint32_t i_closure(const Graph &g, uint32_t s) {
  uint32_t out = s;
  for (int a = 0; a < g.n; ++a) {
    auto sp = g.span(a);
    bool in = true;
    for (int l = sp.first; l <= sp.second; ++l) if (!(s >> l & 1)) { in = false; break; }
    if (in) out |= 1u << (g.n_elec() + a);
  }
  return out;
}

// Deg(s) = -omega(I-closure(s)) / 2 when positive, else c_div; floored at
// d_min.  omega counts momentum powers; the integrand's exponent in the
// Feynman parameters of s is half of it (a parameter scales like the inverse
// square of the momentum through its line), which is the exponent Eq. (1)
// has to match to bound |f|, and what makes Deg fractional (1/2 for a
// single electron line).
inline std::vector<double> deg_table(const Graph &g, double c_div = 0.5, double d_min = 0.05) {
  int N = g.n_lines();
  uint32_t full = (1u << N) - 1;
  std::vector<double> d(size_t(1) << N, 0.0);
  for (uint32_t m = 1; m < full; ++m) {
    int w = -omega(g, i_closure(g, m));
    double v = w > 0 ? 0.5 * double(w) : c_div;
    d[m] = std::max(v, d_min);
  }
  return d;
}

// ---------------------------------------------------------------------------
// UV-divergent subgraphs and forests
// ---------------------------------------------------------------------------
struct Sub {
  int a = 0, b = 0;          // electron lines a..b (inclusive)
  bool se = false;           // self-energy (omega = 1) else vertex-like (0)
  bool has_x = false;        // vertex-like and containing X
  uint32_t lines = 0;        // bitmask over PDF lines
  bool operator==(const Sub &o) const { return a == o.a && b == o.b; }
};

inline std::vector<Sub> divergent_subgraphs(const Graph &g) {
  std::vector<Sub> out;
  for (int a = 0; a < g.n_elec(); ++a)
    for (int b = a; b < g.n_elec(); ++b) {
      if (a == 0 && b == g.n_elec() - 1) continue;
      int lo = a, hi = b + 1;                    // positions lo..hi
      auto inpos = [&](int p) { return p >= lo && p <= hi; };
      int legs = 0;
      std::vector<int> inside;
      for (int p = lo; p <= hi; ++p) {
        if (p == g.e) { ++legs; continue; }
        int ph = g.photon_at(p);
        auto pp = g.ph_pos(ph);
        if (!(inpos(pp.first) && inpos(pp.second))) ++legs;
      }
      if (legs > 1) continue;
      for (int ph = 0; ph < g.n; ++ph) { auto pp = g.ph_pos(ph); if (inpos(pp.first) && inpos(pp.second)) inside.push_back(ph); }
      // 1PI: every electron line of the segment under some internal photon
      bool ok = true;
      for (int l = a; l <= b && ok; ++l) {
        bool cov = false;
        for (int ph : inside) { auto sp = g.span(ph); if (l >= sp.first && l <= sp.second) cov = true; }
        ok = cov;
      }
      if (!ok) continue;
      Sub s; s.a = a; s.b = b; s.se = (legs == 0);
      s.has_x = !s.se && inpos(g.e);
      for (int l = a; l <= b; ++l) s.lines |= 1u << l;
      for (int ph : inside) s.lines |= 1u << (g.n_elec() + ph);
      out.push_back(s);
    }
  return out;
}

inline std::vector<std::vector<Sub>> forests(const Graph &g) {
  auto subs = divergent_subgraphs(g);
  std::vector<std::vector<Sub>> out;
  int m = int(subs.size());
  for (uint32_t mask = 0; mask < (1u << m); ++mask) {
    std::vector<Sub> f;
    for (int i = 0; i < m; ++i) if (mask >> i & 1) f.push_back(subs[i]);
    bool ok = true;
    for (size_t i = 0; i < f.size() && ok; ++i)
      for (size_t j = i + 1; j < f.size() && ok; ++j) {
        uint32_t x = f[i].lines, y = f[j].lines;
        bool nested = ((x & y) == x) || ((x & y) == y);
        if (!(nested || (x & y) == 0)) ok = false;
      }
    if (ok) out.push_back(f);
  }
  // order by size then mask for determinism
  std::stable_sort(out.begin(), out.end(), [](const std::vector<Sub> &x, const std::vector<Sub> &y) { return x.size() < y.size(); });
  return out;
}

}  // namespace qed
