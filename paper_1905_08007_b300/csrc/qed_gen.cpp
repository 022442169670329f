// Integrand code generator (host C++, runs at build time).
//
// For every vertex graph of the requested loop orders it builds the
// forest-like subtraction formula (Sec. 2: linear operators applied to the
// amplitudes of UV-divergent subdiagrams; each graph's contribution is one
// Feynman-parametric integral) and emits straight-line device code for the
// subtracted integrand, templated on the scalar type so that the same source
// serves the FP64 path and the double-double re-evaluation of flagged points
// (Sec. 3: arithmetics of different precisions).
//
// Operator reading (the paper defers the definitions to its references):
//   U on a vertex-like subgraph S: S at zero external momenta, c * gamma_mu;
//   U on a self-energy S: on-shell mass part + (k-slash - m) * slope at k = 0;
//   L on a vertex-like S: on-shell forward vertex constant;
//   A on a vertex-like S containing X: F2(0) of S;
//   A~_G = sum_F (-1)^|F| [ T(F;G) + sum_{G' in F, X in G'} T(F;G') ],
//   T(F;G'): G' gets A, the root G gets (L - U) when G' != G, every element
//   of F strictly containing G' gets L (it is both a link of the infrared
//   chain, L - U, and the ultraviolet counterterm U of the block around it),
//   every other element gets U.
// Every operator value is a block of the same Feynman parameters whose loop
// momenta decouple from the enclosing loops (block-diagonal Lambda).
//
// Integrand of one term (Feynman gauge, m = 1, in units of (alpha/pi)^n):
//   (-1)^n 4^-n sum_{k<n} (-1)^k Gamma(n-k) U^-2 V^(k-n) (2U)^-k
//       sum_{k contractions} prod B_ij * projected Dirac string.
//
// Dirac coefficients: every factor of a string (gamma^mu in the Dirac
// representation, p-slash = gamma^0 in the rest frame, the identity) has one
// non-zero entry per row, so strings are multiplied as (column map, values)
// pairs and projected with trace functionals Tr[W M].
//
// Usage: qed_gen <out.cu> <loop orders...>
#include <atomic>
#include <cmath>
#include <thread>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <set>
#include <sstream>
#include <string>
#include <vector>

#include "qed_graph.hpp"
#include "qed_vm_gen.hpp"

using cd = std::complex<long double>;
using namespace qed;

// ---------------------------------------------------------------------------
// monomial 4x4 matrices
// ---------------------------------------------------------------------------
struct Mono {
  int col[4];
  cd val[4];
};
static Mono mono_identity() { Mono m; for (int r = 0; r < 4; ++r) { m.col[r] = r; m.val[r] = 1.0; } return m; }
// a * b
static Mono mono_mul(const Mono &a, const Mono &b) {
  Mono m;
  for (int r = 0; r < 4; ++r) { int c = a.col[r]; m.col[r] = b.col[c]; m.val[r] = a.val[r] * b.val[c]; }
  return m;
}
static Mono GAM[4];          // gamma^mu
static Mono GAM_LOW[4];      // gamma_mu
static double METRIC[4] = {1, -1, -1, -1};
typedef cd Dense[4][4];
static void to_dense(const Mono &m, Dense &d) {
  for (int r = 0; r < 4; ++r) for (int c = 0; c < 4; ++c) d[r][c] = 0.0;
  for (int r = 0; r < 4; ++r) d[r][m.col[r]] = m.val[r];
}
static void dense_mul(const Dense &a, const Dense &b, Dense &o) {
  Dense t;
  for (int r = 0; r < 4; ++r) for (int c = 0; c < 4; ++c) { cd s = 0; for (int k = 0; k < 4; ++k) s += a[r][k] * b[k][c]; t[r][c] = s; }
  for (int r = 0; r < 4; ++r) for (int c = 0; c < 4; ++c) o[r][c] = t[r][c];
}
// Tr[W M] for dense W, monomial M
static cd tr_wm(const Dense &W, const Mono &M) {
  cd s = 0;
  for (int r = 0; r < 4; ++r) s += W[M.col[r]][r] * M.val[r];
  return s;
}

static void init_gammas() {
  const cd I(0, 1);
  Mono g0; for (int r = 0; r < 4; ++r) { g0.col[r] = r; g0.val[r] = r < 2 ? 1.0 : -1.0; }
  // gamma^k = [[0, s_k], [-s_k, 0]]
  cd s[3][2][2] = {{{0, 1}, {1, 0}}, {{0, -I}, {I, 0}}, {{1, 0}, {0, -1}}};
  GAM[0] = g0;
  for (int k = 0; k < 3; ++k) {
    Mono m;
    for (int r = 0; r < 2; ++r) for (int c = 0; c < 2; ++c)
      if (std::abs(s[k][r][c]) > 0) { m.col[r] = 2 + c; m.val[r] = s[k][r][c]; m.col[2 + r] = c; m.val[2 + r] = -s[k][r][c]; }
    GAM[k + 1] = m;
  }
  for (int mu = 0; mu < 4; ++mu) { GAM_LOW[mu] = GAM[mu]; for (int r = 0; r < 4; ++r) GAM_LOW[mu].val[r] *= METRIC[mu]; }
}

// Trace functionals used by the projections (rest frame, m = 1).
static Dense W_F1;            // (1/4)(1 + gamma^0): charge / on-shell constant / mass part
static Dense W_MAG_G[4];      // magnetic part from G^i (index mu = i)
static Dense W_MAG_H[4][4];   // magnetic part from dG^i/dq^j
static Dense W_UV[4];         // gamma_mu / 16
static Dense W_WF[4];         // gamma^nu / 16
static void init_projectors() {
  const cd I(0, 1);
  Dense one, g0, Pp, Sig[4], gj[4];
  for (int r = 0; r < 4; ++r) for (int c = 0; c < 4; ++c) one[r][c] = (r == c) ? 1.0 : 0.0;
  to_dense(GAM[0], g0);
  for (int r = 0; r < 4; ++r) for (int c = 0; c < 4; ++c) { Pp[r][c] = 0.5L * (one[r][c] + g0[r][c]); W_F1[r][c] = 0.25L * (one[r][c] + g0[r][c]); }
  for (int j = 1; j < 4; ++j) to_dense(GAM[j], gj[j]);
  // Sigma^l = (i/2) eps_ljk gamma^j gamma^k = diag(s_l, s_l)
  for (int l = 1; l < 4; ++l) {
    int j = l % 3 + 1, k = (l + 1) % 3 + 1;
    Dense a, b;
    dense_mul(gj[j], gj[k], a);
    dense_mul(gj[k], gj[j], b);
    for (int r = 0; r < 4; ++r) for (int c = 0; c < 4; ++c) Sig[l][r][c] = 0.5L * I * (a[r][c] - b[r][c]);
  }
  auto eps = [](int i, int j, int l) -> double {
    if (i == j || j == l || i == l) return 0.0;
    int p[3] = {i, j, l};
    int inv = 0;
    for (int x = 0; x < 3; ++x) for (int y = x + 1; y < 3; ++y) if (p[x] > p[y]) ++inv;
    return inv % 2 ? -1.0 : 1.0;
  };
  for (int i = 0; i < 4; ++i) {
    for (int r = 0; r < 4; ++r) for (int c = 0; c < 4; ++c) W_MAG_G[i][r][c] = 0.0;
    for (int j = 0; j < 4; ++j) for (int r = 0; r < 4; ++r) for (int c = 0; c < 4; ++c) W_MAG_H[i][j][r][c] = 0.0;
  }
  // magnetic moment (F1+F2) = (i/6) sum eps_ijl Tr[P+ Sigma^l (H^i_j - [gamma^j, G^i]/4)]
  for (int i = 1; i < 4; ++i)
    for (int j = 1; j < 4; ++j)
      for (int l = 1; l < 4; ++l) {
        double e = eps(i, j, l);
        if (e == 0.0) continue;
        Dense PS, PSg, gPS;
        dense_mul(Pp, Sig[l], PS);
        dense_mul(PS, gj[j], PSg);
        dense_mul(gj[j], PS, gPS);
        for (int r = 0; r < 4; ++r) for (int c = 0; c < 4; ++c) {
          W_MAG_H[i][j][r][c] += (I / 6.0L) * (long double)e * PS[r][c];
          // Tr[PS (-(g M - M g)/4)] = -1/4 (Tr[PS g M] - Tr[g PS M])
          W_MAG_G[i][r][c] += (I / 6.0L) * (long double)e * (-0.25L) * (PSg[r][c] - gPS[r][c]);
        }
      }
  for (int mu = 0; mu < 4; ++mu) {
    Dense d; to_dense(GAM_LOW[mu], d);
    Dense u; to_dense(GAM[mu], u);
    for (int r = 0; r < 4; ++r) for (int c = 0; c < 4; ++c) { W_UV[mu][r][c] = d[r][c] / 16.0L; W_WF[mu][r][c] = u[r][c] / 16.0L; }
  }
}

// ---------------------------------------------------------------------------
// term structure
// ---------------------------------------------------------------------------
enum Kin { KIN_Q, KIN_P, KIN_0, KIN_K };
enum Proj { PR_F2, PR_L, PR_UV, PR_SEMASS, PR_SEWF };

struct Block {
  int a, b;              // electron lines a..b
  bool root, se, has_x;
  Kin kin;
  Proj proj;
  int parent = -1;
  std::vector<int> children;
  bool has_pos(int p) const { return p >= a && p <= b + 1; }
  bool has_line(int l) const { return l >= a && l <= b; }
  int width() const { return b - a; }
};

struct Term {
  int sign;
  std::vector<Block> blocks;     // blocks[0] = root
};

static std::vector<Term> build_terms(const Graph &g) {
  std::vector<Term> out;
  for (auto &F : forests(g)) {
    int fsign = (F.size() % 2) ? -1 : 1;
    std::vector<int> gps = {-1};
    for (size_t i = 0; i < F.size(); ++i) if (F[i].has_x) gps.push_back(int(i));
    for (int gp : gps) {
      // options per element: list of (sign, kin, proj)
      std::vector<std::vector<std::tuple<int, Kin, Proj>>> opts;
      for (size_t i = 0; i < F.size(); ++i) {
        const Sub &s = F[i];
        if (gp >= 0 && int(i) == gp) opts.push_back({{1, KIN_Q, PR_F2}});
        else if (gp >= 0 && (s.lines & F[gp].lines) == F[gp].lines && s.lines != F[gp].lines)
          opts.push_back({{1, KIN_P, PR_L}});
        else if (s.se) opts.push_back({{1, KIN_P, PR_SEMASS}, {1, KIN_K, PR_SEWF}});
        else opts.push_back({{1, KIN_0, PR_UV}});
      }
      std::vector<std::tuple<int, Kin, Proj>> roots;
      if (gp < 0) roots = {{1, KIN_Q, PR_F2}};
      else roots = {{1, KIN_P, PR_L}, {-1, KIN_0, PR_UV}};
      size_t ncomb = 1;
      for (auto &o : opts) ncomb *= o.size();
      for (auto &rt : roots)
        for (size_t c = 0; c < ncomb; ++c) {
          Term t;
          t.sign = fsign * std::get<0>(rt);
          Block r; r.a = 0; r.b = g.n_elec() - 1; r.root = true; r.se = false; r.has_x = true;
          r.kin = std::get<1>(rt); r.proj = std::get<2>(rt);
          t.blocks.push_back(r);
          size_t cc = c;
          for (size_t i = 0; i < F.size(); ++i) {
            auto &o = opts[i][cc % opts[i].size()];
            cc /= opts[i].size();
            Block b; b.a = F[i].a; b.b = F[i].b; b.root = false; b.se = F[i].se; b.has_x = F[i].has_x;
            b.kin = std::get<1>(o); b.proj = std::get<2>(o);
            t.sign *= std::get<0>(o);
            t.blocks.push_back(b);
          }
          // parents
          for (size_t i = 1; i < t.blocks.size(); ++i) {
            int best = 0;
            for (size_t j = 1; j < t.blocks.size(); ++j) {
              if (j == i) continue;
              auto &O = t.blocks[j], &B = t.blocks[i];
              if (O.a <= B.a && B.b <= O.b && O.width() > B.width() && O.width() < t.blocks[best].width()) best = int(j);
            }
            t.blocks[i].parent = best;
            t.blocks[best].children.push_back(int(i));
          }
          for (auto &b : t.blocks)
            std::sort(b.children.begin(), b.children.end(), [&](int x, int y) { return t.blocks[x].a < t.blocks[y].a; });
          out.push_back(t);
        }
    }
  }
  return out;
}

// Item of a block's own Dirac string (increasing position = rightmost first)
enum ItemKind { IT_VTX_PH, IT_VTX_MU, IT_LINE, IT_SEMASS, IT_INS };
struct Item {
  ItemKind kind;
  int photon = -1;       // IT_VTX_PH
  int line = -1;         // IT_LINE: line; IT_INS: entering line
  int child = -1;        // SE child block
};

struct TermInfo {
  const Graph *g;
  Term t;
  std::vector<int> mb_line, mb_ph;
  std::vector<std::vector<int>> eta;       // [line][photon] 0/1 (all 3n lines)
  std::vector<double> alpha, beta, kappa, mass2;
  std::vector<std::vector<Item>> seq;      // per block
};

static int min_block_line(const Term &t, int l) {
  int best = 0;
  for (size_t i = 0; i < t.blocks.size(); ++i)
    if (t.blocks[i].has_line(l) && t.blocks[i].width() < t.blocks[best].width()) best = int(i);
  return best;
}
static int min_block_ph(const Graph &g, const Term &t, int a) {
  auto pp = g.ph_pos(a);
  int best = 0;
  for (size_t i = 0; i < t.blocks.size(); ++i)
    if (t.blocks[i].has_pos(pp.first) && t.blocks[i].has_pos(pp.second) && t.blocks[i].width() < t.blocks[best].width()) best = int(i);
  return best;
}

// label a vertex-like child (or a vertex) carries in block bi: photon id or -1 for mu
static int leg_of_child(const TermInfo &T, int bi, int ci) {
  const Graph &g = *T.g;
  const Block &c = T.t.blocks[ci];
  if (c.has_pos(g.e)) return -1;
  for (int p = c.a; p <= c.b + 1; ++p) {
    int a = g.photon_at(p);
    auto pp = g.ph_pos(a);
    if (!(c.has_pos(pp.first) && c.has_pos(pp.second))) return T.mb_ph[a] == bi ? a : -1;
  }
  fprintf(stderr, "vertex block without leg\n");
  exit(1);
}

static TermInfo analyse(const Graph &g, const Term &t) {
  TermInfo T; T.g = &g; T.t = t;
  int n = g.n, L = g.n_lines();
  for (int l = 0; l < g.n_elec(); ++l) T.mb_line.push_back(min_block_line(t, l));
  for (int a = 0; a < n; ++a) T.mb_ph.push_back(min_block_ph(g, t, a));
  T.eta.assign(L, std::vector<int>(n, 0));
  for (int a = 0; a < n; ++a) {
    auto sp = g.span(a);
    for (int l = sp.first; l <= sp.second; ++l) if (T.mb_line[l] == T.mb_ph[a]) T.eta[l][a] = 1;
    T.eta[g.n_elec() + a][a] = 1;
  }
  T.alpha.assign(L, 0); T.beta.assign(L, 0); T.kappa.assign(L, 0); T.mass2.assign(L, 0);
  for (int l = 0; l < g.n_elec(); ++l) {
    T.mass2[l] = 1.0;
    Kin k = t.blocks[T.mb_line[l]].kin;
    double ax = (l >= g.e) ? 1.0 : 0.0;
    if (k == KIN_Q) { T.alpha[l] = 1.0; T.beta[l] = ax - 0.5; }
    else if (k == KIN_P) T.alpha[l] = 1.0;
    else if (k == KIN_K) T.kappa[l] = 1.0;
  }
  T.seq.resize(t.blocks.size());
  for (size_t bi = 0; bi < t.blocks.size(); ++bi) {
    const Block &B = t.blocks[bi];
    std::map<int, int> ch;
    for (int c : B.children) ch[t.blocks[c].a] = c;
    auto &S = T.seq[bi];
    int v = B.a;
    while (v <= B.b + 1) {
      auto it = ch.find(v);
      if (it != ch.end()) {
        const Block &C = t.blocks[it->second];
        Item I;
        if (C.se) {
          if (C.proj == PR_SEMASS) { I.kind = IT_SEMASS; I.child = it->second; }
          else { I.kind = IT_INS; I.child = it->second; I.line = C.a - 1; }
        } else {
          int lab = leg_of_child(T, int(bi), it->second);
          if (lab < 0) I.kind = IT_VTX_MU; else { I.kind = IT_VTX_PH; I.photon = lab; }
          I.child = it->second;
        }
        S.push_back(I);
        v = C.b + 1;
        if (v <= B.b) { Item li; li.kind = IT_LINE; li.line = v; S.push_back(li); }
        ++v;
        continue;
      }
      Item I;
      if (v == g.e) I.kind = IT_VTX_MU;
      else {
        int a = g.photon_at(v);
        if (T.mb_ph[a] == int(bi)) { I.kind = IT_VTX_PH; I.photon = a; }
        else I.kind = IT_VTX_MU;
      }
      S.push_back(I);
      if (v <= B.b) { Item li; li.kind = IT_LINE; li.line = v; S.push_back(li); }
      ++v;
    }
  }
  return T;
}

// ---------------------------------------------------------------------------
// coefficients of one block for one contraction pattern
// ---------------------------------------------------------------------------
// Momentum factors of a block: IT_LINE and IT_INS items (indices into seq).
// Parts of an uncontracted factor: '1' (identity, -1 for an insertion),
// 'p' (gamma^0, variable A), 'd' (derivative: -gamma^j * C for q, gamma_nu * K
// for k).  Monomial key = bitmask of 'p' factors (over the block's momentum
// factor list) and the derivative factor (-1 = none).
struct MonoKey {
  uint32_t pmask; int deriv;
  bool operator<(const MonoKey &o) const { return pmask != o.pmask ? pmask < o.pmask : deriv < o.deriv; }
};

struct DFS {
  const std::vector<Item> *seq;
  Proj proj;
  bool allow_p, allow_q, allow_k;
  std::vector<int> slot_of_item;          // momentum-factor index or -1
  std::vector<int> pair_partner;          // item -> partner item for contracted / photon pairs, -1
  std::vector<int> pair_alpha;            // chosen alpha per item (filled in DFS)
  std::map<MonoKey, cd> acc;
  std::map<MonoKey, long double> mag;
  int nitems;

  void leaf(const Mono &M, int mu, int dj, uint32_t pm, int dv) {
    cd v = 0;
    switch (proj) {
      case PR_F2:
        if (dv < 0) { if (mu == 0) v = -tr_wm(W_F1, M); else v = tr_wm(W_MAG_G[mu], M); }
        else { if (mu > 0) v = tr_wm(W_MAG_H[mu][dj], M); }
        break;
      case PR_L: if (mu == 0 && dv < 0) v = tr_wm(W_F1, M); break;
      case PR_UV: if (dv < 0) v = tr_wm(W_UV[mu], M); break;
      case PR_SEMASS: if (dv < 0) v = tr_wm(W_F1, M); break;
      case PR_SEWF: if (dv >= 0) v = tr_wm(W_WF[dj], M); break;
    }
    if (std::abs(v) > 0) { acc[MonoKey{pm, dv}] += v; mag[MonoKey{pm, dv}] += std::abs(v); }
  }
  // t: current item, M: product of items < t (rightmost first), mu/dj state
  void go(int t, const Mono &M, int mu, int dj, uint32_t pm, int dv) {
    if (t == nitems) { leaf(M, mu, dj, pm, dv); return; }
    const Item &I = (*seq)[t];
    auto push = [&](const Mono &F, int mu2, int dj2, uint32_t pm2, int dv2) {
      go(t + 1, mono_mul(F, M), mu2, dj2, pm2, dv2);
    };
    if (pair_partner[t] >= 0) {            // contracted gamma slot
      int p = pair_partner[t];
      if (p > t) {
        for (int a = 0; a < 4; ++a) { pair_alpha[t] = a; push(GAM[a], mu, dj, pm, dv); }
      } else push(GAM_LOW[pair_alpha[p]], mu, dj, pm, dv);
      return;
    }
    switch (I.kind) {
      case IT_VTX_MU:
        if (mu >= 0) { fprintf(stderr, "two free indices\n"); exit(1); }
        for (int m = 0; m < 4; ++m) push(GAM[m], m, dj, pm, dv);
        return;
      case IT_SEMASS:
        push(mono_identity(), mu, dj, pm, dv);
        return;
      case IT_LINE:
      case IT_INS: {
        int f = slot_of_item[t];
        const double sgn = (I.kind == IT_INS) ? -1.0 : 1.0;
        if (allow_p) {
          // (A pslash + 1) = (1+A) P+ + (1-A) P-;  (A pslash - 1) = -(1-A) P+ - (1+A) P-
          // bit 2f: factor (1 + A_f), bit 2f+1: factor (1 - A_f)
          Mono pp, pmn;
          for (int r = 0; r < 4; ++r) { pp.col[r] = r; pmn.col[r] = r; pp.val[r] = r < 2 ? sgn : 0.0; pmn.val[r] = r < 2 ? 0.0 : sgn; }
          const uint32_t bp = (I.kind == IT_INS) ? (1u << (2 * f + 1)) : (1u << (2 * f));
          const uint32_t bm = (I.kind == IT_INS) ? (1u << (2 * f)) : (1u << (2 * f + 1));
          push(pp, mu, dj, pm | bp, dv);
          push(pmn, mu, dj, pm | bm, dv);
        } else {
          Mono one = mono_identity();
          for (int r = 0; r < 4; ++r) one.val[r] = sgn;
          push(one, mu, dj, pm, dv);
        }
        if (dv < 0 && allow_q)
          for (int j = 1; j < 4; ++j) { Mono m = GAM[j]; for (int r = 0; r < 4; ++r) m.val[r] = -m.val[r]; push(m, mu, j, pm, f); }
        if (dv < 0 && allow_k)
          for (int nu = 0; nu < 4; ++nu) push(GAM_LOW[nu], mu, nu, pm, f);
        return;
      }
      default: break;
    }
    fprintf(stderr, "bad item\n");
    exit(1);
  }
};

// The same sum as a transfer-matrix recursion over the items: every branch
// choice (the Lorentz index of an open pair, the free index mu, a factor's
// P+/P- part or derivative) is part of a state key, and the partial product
// of all branches with the same key is kept as one dense matrix.  Closing a
// pair drops its index from the key, which merges the branches that differed
// only there, so the work grows with the number of pairs open at a time
// instead of with all of them.  Every factor's non-zero entries are 1, -1, i
// or -i, so the partial products have Gaussian-integer entries, exact in
// double; only the final trace with the projector rounds.  Items other than
// the closing one of a pair give every state distinct successor keys, so
// only closing items need a lookup.
struct DP {
  const std::vector<Item> *seq;
  Proj proj;
  bool allow_p, allow_q, allow_k;
  std::vector<int> slot_of_item;          // momentum-factor index or -1
  std::vector<int> pair_partner;          // partner item of a photon or contracted pair, -1
  std::map<MonoKey, cd> acc;
  std::map<MonoKey, long double> mag;

  // key: bits 0-23 the alpha of open pairs (2 bits per pair id), 24-26 mu+1,
  // 27-29 dj+1, 30-34 dv+1, 35-63 the P+/P- mask (2 bits per factor)
  static constexpr int MU_SH = 24, DJ_SH = 27, DV_SH = 30, PM_SH = 35;
  struct St { double re[4][4], im[4][4]; };
  std::vector<uint64_t> keys, nkeys;
  std::vector<St> st, nst;
  // open-addressing index of the next item's states (closing items only)
  std::vector<uint64_t> hkey;
  std::vector<int> hval;
  size_t hmask = 0;
  bool merging = false;

  void reset_index(size_t expect) {
    size_t cap = 64;
    while (cap < 2 * expect) cap <<= 1;
    if (hkey.size() < cap) { hkey.assign(cap, 0); hval.assign(cap, -1); }
    else std::fill(hval.begin(), hval.begin() + cap, -1);
    hmask = cap - 1;
  }
  // the state of `key` and whether it already existed
  St &slot(uint64_t key, bool &existed) {
    existed = false;
    if (!merging) { nkeys.push_back(key); nst.emplace_back(); return nst.back(); }
    for (size_t h = (key * 0x9E3779B97F4A7C15ull) >> 17;; ++h) {
      const size_t i = h & hmask;
      if (hval[i] < 0) {
        hkey[i] = key;
        hval[i] = int(nkeys.size());
        nkeys.push_back(key);
        nst.emplace_back();
        return nst.back();
      }
      if (hkey[i] == key) { existed = true; return nst[hval[i]]; }
    }
  }
  // dst (+)= F * src (F monomial with entries in {0, +-1, +-i}); a new
  // state is written, an existing one accumulated
  void push(const Mono &F, const St &src, uint64_t key) {
    bool existed;
    St &d = slot(key, existed);
    if (!existed) {
      for (int r = 0; r < 4; ++r) {
        const double vr = double(F.val[r].real()), vi = double(F.val[r].imag());
        const int c0 = F.col[r];
        for (int c = 0; c < 4; ++c) {
          const double x = src.re[c0][c], y = src.im[c0][c];
          d.re[r][c] = vr * x - vi * y;
          d.im[r][c] = vr * y + vi * x;
        }
      }
      return;
    }
    for (int r = 0; r < 4; ++r) {
      const long double vr = F.val[r].real(), vi = F.val[r].imag();
      const int c0 = F.col[r];
      if (vi == 0.0L) {
        if (vr == 0.0L) continue;
        if (vr > 0) for (int c = 0; c < 4; ++c) { d.re[r][c] += src.re[c0][c]; d.im[r][c] += src.im[c0][c]; }
        else for (int c = 0; c < 4; ++c) { d.re[r][c] -= src.re[c0][c]; d.im[r][c] -= src.im[c0][c]; }
      } else if (vi > 0) {       // i (x + i y) = -y + i x
        for (int c = 0; c < 4; ++c) { d.re[r][c] -= src.im[c0][c]; d.im[r][c] += src.re[c0][c]; }
      } else {
        for (int c = 0; c < 4; ++c) { d.re[r][c] += src.im[c0][c]; d.im[r][c] -= src.re[c0][c]; }
      }
    }
  }
  static cd tr_wd(const Dense &W, const St &M) {
    cd s = 0;
    for (int r = 0; r < 4; ++r) for (int k = 0; k < 4; ++k) s += W[r][k] * cd(M.re[k][r], M.im[k][r]);
    return s;
  }
  // bound on the rounding of tr_wd: sum of the absolute values of its terms
  static long double tr_abs(const Dense &W, const St &M) {
    long double s = 0;
    for (int r = 0; r < 4; ++r)
      for (int k = 0; k < 4; ++k) s += std::abs(W[r][k]) * std::abs(cd(M.re[k][r], M.im[k][r]));
    return s;
  }

  void run() {
    const int nitems = int(seq->size());
    std::vector<int> pid(nitems, -1);
    int np = 0;
    for (int t = 0; t < nitems; ++t) if (pair_partner[t] > t) pid[t] = np++;
    if (np > 12) { fprintf(stderr, "too many open pairs\n"); exit(1); }
    keys.assign(1, 0ull);
    st.assign(1, St{});
    memset(&st[0], 0, sizeof(St));
    for (int r = 0; r < 4; ++r) st[0].re[r][r] = 1.0;
    for (int t = 0; t < nitems; ++t) {
      const Item &I = (*seq)[t];
      nkeys.clear(); nst.clear();
      merging = pair_partner[t] >= 0 && pair_partner[t] < t;
      if (merging) reset_index(keys.size());
      nkeys.reserve(keys.size() * 4); nst.reserve(keys.size() * 4);
      for (size_t si = 0; si < keys.size(); ++si) {
        const uint64_t k = keys[si];
        const St &s = st[si];
        const int mu = int((k >> MU_SH) & 7) - 1;
        const int dv = int((k >> DV_SH) & 31) - 1;
        if (pair_partner[t] >= 0) {
          const int p = pair_partner[t];
          if (p > t) {
            for (int a = 0; a < 4; ++a) push(GAM[a], s, k | (uint64_t(a) << (2 * pid[t])));
          } else {
            const int a = int((k >> (2 * pid[p])) & 3);
            push(GAM_LOW[a], s, k & ~(3ull << (2 * pid[p])));
          }
          continue;
        }
        switch (I.kind) {
          case IT_VTX_MU:
            if (mu >= 0) { fprintf(stderr, "two free indices\n"); exit(1); }
            // the on-shell constant L projects on mu = 0 only
            for (int m = 0; m < 4; ++m) {
              if (proj == PR_L && m != 0) continue;
              push(GAM[m], s, (k & ~(7ull << MU_SH)) | (uint64_t(m + 1) << MU_SH));
            }
            break;
          case IT_SEMASS:
            push(mono_identity(), s, k);
            break;
          case IT_LINE:
          case IT_INS: {
            const int f = slot_of_item[t];
            const double sgn = (I.kind == IT_INS) ? -1.0 : 1.0;
            if (allow_p) {
              // (A pslash + 1) = (1+A) P+ + (1-A) P-;  (A pslash - 1) = -(1-A) P+ - (1+A) P-
              // mask bit 2f: factor (1 + A_f), bit 2f+1: factor (1 - A_f)
              Mono pp, pmn;
              for (int r = 0; r < 4; ++r) { pp.col[r] = r; pmn.col[r] = r; pp.val[r] = r < 2 ? sgn : 0.0; pmn.val[r] = r < 2 ? 0.0 : sgn; }
              const uint64_t bp = (I.kind == IT_INS) ? (1ull << (PM_SH + 2 * f + 1)) : (1ull << (PM_SH + 2 * f));
              const uint64_t bm = (I.kind == IT_INS) ? (1ull << (PM_SH + 2 * f)) : (1ull << (PM_SH + 2 * f + 1));
              push(pp, s, k | bp);
              push(pmn, s, k | bm);
            } else {
              Mono one = mono_identity();
              for (int r = 0; r < 4; ++r) one.val[r] = sgn;
              push(one, s, k);
            }
            const uint64_t kd = (k & ~((7ull << DJ_SH) | (31ull << DV_SH))) | (uint64_t(f + 1) << DV_SH);
            if (dv < 0 && allow_q)
              for (int j = 1; j < 4; ++j) {
                Mono m = GAM[j];
                for (int r = 0; r < 4; ++r) m.val[r] = -m.val[r];
                push(m, s, kd | (uint64_t(j + 1) << DJ_SH));
              }
            if (dv < 0 && allow_k)
              for (int nu = 0; nu < 4; ++nu) push(GAM_LOW[nu], s, kd | (uint64_t(nu + 1) << DJ_SH));
            break;
          }
          default:
            fprintf(stderr, "bad item\n");
            exit(1);
        }
      }
      keys.swap(nkeys);
      st.swap(nst);
    }
    for (size_t si = 0; si < keys.size(); ++si) {
      const uint64_t k = keys[si];
      const int mu = int((k >> MU_SH) & 7) - 1;
      const int dj = int((k >> DJ_SH) & 7) - 1;
      const int dv = int((k >> DV_SH) & 31) - 1;
      const uint32_t pm = uint32_t(k >> PM_SH);
      const Dense *W = nullptr;
      long double sg = 1.0L;
      switch (proj) {
        case PR_F2:
          if (dv < 0) { if (mu == 0) { W = &W_F1; sg = -1.0L; } else if (mu > 0) W = &W_MAG_G[mu]; }
          else if (mu > 0) W = &W_MAG_H[mu][dj];
          break;
        case PR_L: if (mu == 0 && dv < 0) W = &W_F1; break;
        case PR_UV: if (dv < 0 && mu >= 0) W = &W_UV[mu]; break;
        case PR_SEMASS: if (dv < 0) W = &W_F1; break;
        case PR_SEWF: if (dv >= 0) W = &W_WF[dj]; break;
      }
      if (!W) continue;
      const cd v = cd(sg) * tr_wd(*W, st[si]);
      if (std::abs(v) > 0) {
        acc[MonoKey{pm, dv}] += v;
        mag[MonoKey{pm, dv}] += tr_abs(*W, st[si]);
      }
    }
  }
};

// ---------------------------------------------------------------------------
// code emission
// ---------------------------------------------------------------------------
static std::string dstr(double x) {
  char b[64];
  snprintf(b, sizeof b, "%.17g", x);
  std::string s = b;
  if (s.find('.') == std::string::npos && s.find('e') == std::string::npos) s += ".0";
  return s;
}

// Dirac coefficients are rationals whose denominators divide 2^12 * 3;
// summing them (in long double) leaves rounding noise relative to the
// magnitude of the summed contributions, removed here.
static double snap(long double c, long double mag) {
  const long double den = 4096.0L * 3.0L;
  const long double r = std::round(c * den);
  const long double tol = 1e-6L + 1e-14L * mag * den;
  if (std::abs(c * den - r) < tol) return double(r / den);
  fprintf(stderr, "coefficient %.17Lg (magnitude %.3Lg) is not a small rational\n", c, mag);
  exit(1);
}

struct Emitter {
  std::ostringstream os;
  int tmp = 0;
  std::string fresh(const char *p) { return std::string(p) + std::to_string(tmp++); }
  // polynomials already emitted in this graph's function, by content key:
  // forest terms with the same block structure share U, 1/U, B_ij, and with
  // the same kinematics also (1 +- A), C, K and V
  std::map<std::string, std::string> cache;
};

// Emit a sum of z's (as R expression); returns "" if empty
static std::string zsum(const std::vector<int> &ls) {
  if (ls.empty()) return "";
  std::string s;
  for (size_t i = 0; i < ls.size(); ++i) s += (i ? " + z[" : "z[") + std::to_string(ls[i]) + "]";
  return s;
}

// ---------------------------------------------------------------------------
// symbolic polynomials in the Feynman parameters (dyadic-rational
// coefficients, exact in binary floating point)
// ---------------------------------------------------------------------------
struct Poly {
  std::map<std::vector<int>, double> t;     // sorted variable multiset -> coefficient
  static Poly var(int l) { Poly p; p.t[{l}] = 1.0; return p; }
  static Poly cst(double c) { Poly p; if (c != 0.0) p.t[{}] = c; return p; }
  bool zero() const { return t.empty(); }
  void clean() { for (auto it = t.begin(); it != t.end();) { if (it->second == 0.0) it = t.erase(it); else ++it; } }
  Poly operator+(const Poly &o) const { Poly r = *this; for (auto &kv : o.t) r.t[kv.first] += kv.second; r.clean(); return r; }
  Poly operator-(const Poly &o) const { Poly r = *this; for (auto &kv : o.t) r.t[kv.first] -= kv.second; r.clean(); return r; }
  Poly operator*(double c) const { Poly r; if (c == 0.0) return r; for (auto &kv : t) r.t[kv.first] = kv.second * c; return r; }
  Poly operator*(const Poly &o) const {
    Poly r;
    for (auto &a : t) for (auto &b : o.t) {
      std::vector<int> m = a.first;
      m.insert(m.end(), b.first.begin(), b.first.end());
      std::sort(m.begin(), m.end());
      r.t[m] += a.second * b.second;
    }
    r.clean();
    return r;
  }
  // nested (Horner-like) form over named variables (names[v] replaces z[v])
  std::string horner_named(const std::vector<std::string> &names) const {
    if (t.empty()) return "R(0.0)";
    std::map<int, int> freq;
    for (auto &kv : t) { std::set<int> u(kv.first.begin(), kv.first.end()); for (int v : u) ++freq[v]; }
    if (freq.empty()) return "R(" + dstr(t.begin()->second) + ")";
    int best = -1, bc = 0;
    for (auto &kv : freq) if (kv.second > bc) { bc = kv.second; best = kv.first; }
    Poly with, without;
    for (auto &kv : t) {
      auto it = std::find(kv.first.begin(), kv.first.end(), best);
      if (it == kv.first.end()) { without.t[kv.first] = kv.second; continue; }
      std::vector<int> m = kv.first;
      m.erase(m.begin() + (it - kv.first.begin()));
      with.t[m] = kv.second;
    }
    const std::string &zv = names[best];
    std::string inner;
    if (with.t.size() == 1 && with.t.begin()->first.empty()) {
      double c = with.t.begin()->second;
      inner = (c == 1.0) ? zv : "R(" + dstr(c) + ") * " + zv;
    } else {
      inner = zv + " * (" + with.horner_named(names) + ")";
    }
    if (without.zero()) return inner;
    return inner + " + " + without.horner_named(names);
  }
  // nested (Horner-like) form: factor out the most frequent variable
  std::string horner() const {
    if (t.empty()) return "R(0.0)";
    std::map<int, int> freq;
    for (auto &kv : t) { std::set<int> u(kv.first.begin(), kv.first.end()); for (int v : u) ++freq[v]; }
    if (freq.empty()) return "R(" + dstr(t.begin()->second) + ")";
    int best = -1, bc = 0;
    for (auto &kv : freq) if (kv.second > bc) { bc = kv.second; best = kv.first; }
    Poly with, without;
    for (auto &kv : t) {
      auto it = std::find(kv.first.begin(), kv.first.end(), best);
      if (it == kv.first.end()) { without.t[kv.first] = kv.second; continue; }
      std::vector<int> m = kv.first;
      m.erase(m.begin() + (it - kv.first.begin()));
      with.t[m] = kv.second;
    }
    std::string zv = "z[" + std::to_string(best) + "]";
    std::string inner;
    if (with.t.size() == 1 && with.t.begin()->first.empty()) {
      double c = with.t.begin()->second;
      inner = (c == 1.0) ? zv : "R(" + dstr(c) + ") * " + zv;
    } else {
      inner = zv + " * (" + with.horner() + ")";
    }
    if (without.zero()) return inner;
    return inner + " + " + without.horner();
  }
};

static Poly det_poly(const std::vector<std::vector<Poly>> &m) {
  const int n = int(m.size());
  if (n == 0) return Poly::cst(1.0);
  if (n == 1) return m[0][0];
  Poly r;
  for (int c = 0; c < n; ++c) {
    if (m[0][c].zero()) continue;
    std::vector<std::vector<Poly>> sub;
    for (int i = 1; i < n; ++i) {
      std::vector<Poly> row;
      for (int j = 0; j < n; ++j) if (j != c) row.push_back(m[i][j]);
      sub.push_back(row);
    }
    Poly d = m[0][c] * det_poly(sub);
    r = (c % 2) ? r - d : r + d;
  }
  return r;
}

// (-1)^(r+c) det(m without row r and column c)
static Poly cofactor_poly(const std::vector<std::vector<Poly>> &m, int r, int c) {
  const int n = int(m.size());
  std::vector<std::vector<Poly>> sub;
  for (int i = 0; i < n; ++i) {
    if (i == r) continue;
    std::vector<Poly> row;
    for (int j = 0; j < n; ++j) if (j != c) row.push_back(m[i][j]);
    sub.push_back(row);
  }
  Poly d = det_poly(sub);
  return ((r + c) % 2) ? d * -1.0 : d;
}

struct GenStats { long terms = 0, monos = 0; };

// Emits code computing one term's value into variable `out` (declared here).
static void emit_term(Emitter &E, const TermInfo &T, const std::string &out, GenStats &st) {
  const Graph &g = *T.g;
  int n = g.n, L = g.n_lines();
  auto &os = E.os;
  std::string P = E.fresh("t");
  // Graph polynomials, expanded symbolically so that every cancellation
  // between monomials happens here, exactly, and the device evaluates
  // polynomials whose terms do not cancel (U, B_ij, U V have non-negative
  // coefficients; U A_l too on lines carrying the external momentum).
  std::vector<std::vector<Poly>> lam(n, std::vector<Poly>(n));
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b)
      for (int l = 0; l < L; ++l) if (T.eta[l][a] && T.eta[l][b]) lam[a][b] = lam[a][b] + Poly::var(l);
  Poly Up = det_poly(lam);
  std::vector<std::vector<Poly>> adjp(n, std::vector<Poly>(n));
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) adjp[a][b] = cofactor_poly(lam, b, a);
  std::string eta_key;
  for (int l = 0; l < L; ++l) { for (int a = 0; a < n; ++a) eta_key += char('0' + T.eta[l][a]); eta_key += '|'; }
  auto vec_key = [](const std::vector<double> &v) { std::string k; for (double x : v) k += dstr(x) + ","; return k; };
  std::string U, iU;
  {
    auto it = E.cache.find("U" + eta_key);
    if (it != E.cache.end()) { U = it->second; iU = it->second + "_inv"; }
    else {
      U = P + "_U"; iU = U + "_inv";
      os << "    const R " << U << " = " << Up.horner() << ";\n";
      os << "    const R " << iU << " = R(1.0) / " << U << ";\n";
      E.cache["U" + eta_key] = U;
    }
  }
  os << "    const R& " << P << "_iU = " << iU << ";\n";
  auto Jpoly = [&](const std::vector<double> &coef) {
    std::vector<Poly> J(n);
    for (int a = 0; a < n; ++a)
      for (int l = 0; l < L; ++l) if (T.eta[l][a] && coef[l] != 0.0) J[a] = J[a] + Poly::var(l) * coef[l];
    return J;
  };
  auto Xpoly = [&](const std::vector<Poly> &J) {
    std::vector<Poly> X(n);
    for (int a = 0; a < n; ++a)
      for (int b = 0; b < n; ++b) X[a] = X[a] + adjp[a][b] * J[b];
    return X;
  };
  auto Jp = Jpoly(T.alpha), Jq = Jpoly(T.beta), Jk = Jpoly(T.kappa);
  auto Xp = Xpoly(Jp), Xq = Xpoly(Jq), Xk = Xpoly(Jk);
  std::vector<std::string> A(L), C(L), K(L);
  // Q coefficient of line l times U: coef_l U - eta_l . adj . J
  auto emitQ = [&](const std::vector<double> &coef, const std::vector<Poly> &X, int l, const char *tag) -> std::string {
    Poly q = Up * coef[l];
    for (int a = 0; a < n; ++a) if (T.eta[l][a]) q = q - X[a];
    if (q.zero()) return "";
    const std::string key = std::string(tag) + eta_key + vec_key(coef) + std::to_string(l);
    auto it = E.cache.find(key);
    if (it != E.cache.end()) return it->second;
    std::string v = P + "_" + tag + std::to_string(l);
    os << "    const R " << v << " = (" << q.horner() << ") * " << P << "_iU;\n";
    E.cache[key] = v;
    return v;
  };
  for (int l = 0; l < g.n_elec(); ++l) {
    C[l] = emitQ(T.beta, Xq, l, "Cq");
    K[l] = emitQ(T.kappa, Xk, l, "Kk");
  }
  // V = sum_{electrons without external momentum} z + Jp . adj . Jp / U
  std::string V;
  {
    const std::string key = "V" + eta_key + vec_key(T.alpha);
    auto it = E.cache.find(key);
    if (it != E.cache.end()) V = it->second;
    else {
      V = P + "_V";
      Poly uv;
      for (int l = 0; l < g.n_elec(); ++l) if (T.alpha[l] == 0.0) uv = uv + Up * Poly::var(l);
      for (int a = 0; a < n; ++a) uv = uv + Jp[a] * Xp[a];
      os << "    const R " << V << " = (" << uv.horner() << ") * " << P << "_iU;\n";
      os << "    const R " << V << "_inv = R(1.0) / " << V << ";\n";
      E.cache[key] = V;
    }
  }
  // (1 + A_l) and (1 - A_l), expanded symbolically: (U +- U A_l) / U
  std::map<std::pair<int, int>, std::string> onepm_cache;
  auto onepm = [&](int l, int minus) -> std::string {
    auto key = std::make_pair(l, minus);
    auto it = onepm_cache.find(key);
    if (it != onepm_cache.end()) return it->second;
    const std::string gkey = std::string(minus ? "Bm" : "Bp") + eta_key + vec_key(T.alpha) + std::to_string(l);
    auto git = E.cache.find(gkey);
    if (git != E.cache.end()) { onepm_cache[key] = git->second; return git->second; }
    Poly q = Up * T.alpha[l];
    for (int a = 0; a < n; ++a) if (T.eta[l][a]) q = q - Xp[a];
    Poly w = minus ? Up - q : Up + q;
    std::string v = P + (minus ? "_Bm" : "_Bp") + std::to_string(l);
    os << "    const R " << v << " = (" << w.horner() << ") * " << P << "_iU;\n";
    onepm_cache[key] = v;
    E.cache[gkey] = v;
    return v;
  };
  // B_ij on demand
  std::map<std::pair<int, int>, std::string> Bc;
  auto Bij = [&](int i, int j) -> std::string {
    if (i > j) std::swap(i, j);
    auto key = std::make_pair(i, j);
    auto it = Bc.find(key);
    if (it != Bc.end()) return it->second;
    Poly bp;
    for (int a = 0; a < n; ++a) for (int b = 0; b < n; ++b)
      if (T.eta[i][a] && T.eta[j][b]) bp = bp + adjp[a][b];
    std::string v;
    if (!bp.zero()) {
      const std::string gkey = "B" + eta_key + std::to_string(i) + "_" + std::to_string(j);
      auto git = E.cache.find(gkey);
      if (git != E.cache.end()) v = git->second;
      else {
        v = P + "_B" + std::to_string(i) + "_" + std::to_string(j);
        os << "    const R " << v << " = " << bp.horner() << ";\n";
        E.cache[gkey] = v;
      }
    }
    Bc[key] = v;
    return v;
  };
  // |A|, |C|, |K| in FP32 for the condition estimate (all lie in [-1, 1]
  // up to O(1) factors, so single precision has the range and accuracy an
  // estimate needs; FP32 is the cheap pipe)
  auto fabsvar = [&](const std::string &v) -> std::string {
    auto it = E.cache.find("fa:" + v);
    if (it != E.cache.end()) return it->second;
    std::string fv = "fa_" + v;
    os << "    const float " << fv << " = fabsf(float(to_double(" << v << ")));\n";
    E.cache["fa:" + v] = fv;
    return fv;
  };
  // block values: recursive, returns (value, absolute-sum) variable names per k
  typedef std::pair<std::vector<std::string>, std::vector<std::string>> VA;
  std::function<VA(int)> block_val = [&](int bi) -> VA {
    const Block &B = T.t.blocks[bi];
    const auto &seq = T.seq[bi];
    std::vector<VA> childv;
    for (int c : B.children) childv.push_back(block_val(c));
    // momentum factors
    std::vector<int> mom_items;
    std::vector<int> mom_line;   // line whose eta/A/C/K the factor uses
    for (size_t t = 0; t < seq.size(); ++t)
      if (seq[t].kind == IT_LINE || seq[t].kind == IT_INS) { mom_items.push_back(int(t)); mom_line.push_back(seq[t].line); }
    std::vector<std::pair<int, int>> ph_pairs;
    {
      std::map<int, std::vector<int>> byph;
      for (size_t t = 0; t < seq.size(); ++t) if (seq[t].kind == IT_VTX_PH) byph[seq[t].photon].push_back(int(t));
      for (auto &kv : byph) {
        if (kv.second.size() != 2) { fprintf(stderr, "unpaired photon\n"); exit(1); }
        ph_pairs.push_back({kv.second[0], kv.second[1]});
      }
    }
    int m = int(mom_items.size());
    // enumerate pairings of momentum factors
    std::vector<std::vector<std::pair<int, int>>> pats;
    std::function<void(std::vector<int>, std::vector<std::pair<int, int>>)> rec =
        [&](std::vector<int> rest, std::vector<std::pair<int, int>> cur) {
          if (rest.size() < 2) { pats.push_back(cur); return; }
          int f = rest[0];
          std::vector<int> r1(rest.begin() + 1, rest.end());
          rec(r1, cur);
          for (size_t i = 0; i < r1.size(); ++i) {
            std::vector<int> r2;
            for (size_t j = 0; j < r1.size(); ++j) if (j != i) r2.push_back(r1[j]);
            auto c2 = cur; c2.push_back({f, r1[i]});
            rec(r2, c2);
          }
        };
    std::vector<int> all(m);
    for (int i = 0; i < m; ++i) all[i] = i;
    rec(all, {});
    std::map<int, std::string> ownk;    // k -> accumulated expression variable
    std::map<int, std::string> ownk_abs;  // k -> accumulated absolute sum (double)
    for (auto &pat : pats) {
      // B product
      std::string bprod;
      bool zero = false;
      for (auto &pr : pat) {
        std::string b = Bij(mom_line[pr.first], mom_line[pr.second]);
        if (b.empty()) { zero = true; break; }
        bprod += (bprod.empty() ? "" : " * ") + b;
      }
      if (zero) continue;
      DFS D;
      D.seq = &seq; D.proj = B.proj; D.nitems = int(seq.size());
      D.allow_p = (B.kin == KIN_Q || B.kin == KIN_P);
      D.allow_q = (B.proj == PR_F2);
      D.allow_k = (B.proj == PR_SEWF);
      D.slot_of_item.assign(seq.size(), -1);
      for (int i = 0; i < m; ++i) D.slot_of_item[mom_items[i]] = i;
      D.pair_partner.assign(seq.size(), -1);
      D.pair_alpha.assign(seq.size(), 0);
      for (auto &pp : ph_pairs) { D.pair_partner[pp.first] = pp.second; D.pair_partner[pp.second] = pp.first; }
      for (auto &pr : pat) { int a = mom_items[pr.first], b = mom_items[pr.second]; D.pair_partner[a] = b; D.pair_partner[b] = a; }
      if (getenv("QED_GEN_DFS")) D.go(0, mono_identity(), -1, -1, 0u, -1);
      else {
        // one recursion object per thread: its state buffers keep their
        // capacity from run to run
        static thread_local DP Q;
        Q.acc.clear();
        Q.mag.clear();
        Q.seq = D.seq; Q.proj = D.proj; Q.allow_p = D.allow_p; Q.allow_q = D.allow_q; Q.allow_k = D.allow_k;
        Q.slot_of_item = D.slot_of_item; Q.pair_partner = D.pair_partner;
        Q.run();
        D.acc.swap(Q.acc);
        D.mag.swap(Q.mag);
      }
      std::string poly, apoly;
      Poly vpoly;                               // value polynomial over named factors
      std::vector<std::string> vnames;
      std::map<std::string, int> vid;
      auto var_id = [&](const std::string &nm) {
        auto it = vid.find(nm);
        if (it != vid.end()) return it->second;
        vid[nm] = int(vnames.size());
        vnames.push_back(nm);
        return int(vnames.size()) - 1;
      };
      for (auto &kv : D.acc) {
        cd c = kv.second;
        if (std::abs(c.imag()) > 1e-9L * (1 + std::abs(c.real()) + D.mag[kv.first])) { fprintf(stderr, "complex coefficient %Lg %Lg\n", c.real(), c.imag()); exit(1); }
        double cr = snap(c.real(), D.mag[kv.first]);
        if (cr == 0.0) continue;
        std::string mono, amono;
        std::vector<int> mids;
        for (int f = 0; f < m; ++f)
          for (int pmn = 0; pmn < 2; ++pmn)
            if (kv.first.pmask >> (2 * f + pmn) & 1) {
              const std::string v = onepm(mom_line[f], pmn);
              mono += " * " + v;
              amono += " * " + fabsvar(v);
              mids.push_back(var_id(v));
            }
        if (kv.first.deriv >= 0) {
          int f = kv.first.deriv;
          const std::string &v = (B.proj == PR_F2) ? C[mom_line[f]] : K[mom_line[f]];
          if (v.empty()) continue;
          mono += " * " + v;
          amono += " * " + fabsvar(v);
          mids.push_back(var_id(v));
        }
        poly += (poly.empty() ? "R(" : " + R(") + dstr(cr) + ")" + mono;
        std::sort(mids.begin(), mids.end());
        vpoly.t[mids] += cr;
        apoly += std::string(apoly.empty() ? "" : " + ") + dstr(std::abs(cr)) + "f" + amono;
        ++st.monos;
      }
      if (poly.empty()) continue;
      int k = int(pat.size());
      std::string var = P + "_b" + std::to_string(bi) + "k" + std::to_string(k);
      vpoly.clean();
      if (!vpoly.zero()) poly = vpoly.horner_named(vnames);
      std::string contrib = bprod.empty() ? "(" + poly + ")" : bprod + " * (" + poly + ")";
      std::string acontrib = bprod.empty() ? "double(" + apoly + ")" : "fabs(to_double(" + bprod + ")) * double(" + apoly + ")";
      std::string avar = var + "_a";
      if (!ownk.count(k)) {
        os << "    R " << var << " = " << contrib << ";\n";
        os << "    double " << avar << " = " << acontrib << ";\n";
        ownk[k] = var; ownk_abs[k] = avar;
      } else {
        os << "    " << var << " = " << var << " + " << contrib << ";\n";
        os << "    " << avar << " = " << avar << " + " << acontrib << ";\n";
      }
    }
    int kmax = ownk.empty() ? 0 : ownk.rbegin()->first;
    std::vector<std::string> vals(kmax + 1), avals(kmax + 1);
    for (int k = 0; k <= kmax; ++k) { vals[k] = ownk.count(k) ? ownk[k] : ""; avals[k] = ownk_abs.count(k) ? ownk_abs[k] : ""; }
    for (auto &cva : childv) {
      const auto &cv = cva.first, &ca = cva.second;
      std::vector<std::string> nv(vals.size() + cv.size() - 1), na(vals.size() + cv.size() - 1);
      for (size_t i = 0; i < vals.size(); ++i) for (size_t j = 0; j < cv.size(); ++j) {
        if (vals[i].empty() || cv[j].empty()) continue;
        std::string v = P + "_c" + std::to_string(bi) + "_" + std::to_string(E.tmp++);
        os << "    const R " << v << " = " << vals[i] << " * " << cv[j] << ";\n";
        os << "    const double " << v << "_a = " << avals[i] << " * " << ca[j] << ";\n";
        nv[i + j] = nv[i + j].empty() ? v : "(" + nv[i + j] + " + " + v + ")";
        na[i + j] = na[i + j].empty() ? v + "_a" : "(" + na[i + j] + " + " + v + "_a)";
      }
      vals = nv;
      avals = na;
    }
    return VA(vals, avals);
  };
  auto va = block_val(0);
  auto &vals = va.first;
  auto &avals = va.second;
  // combine: (-1)^n 4^-n sum_k (-1)^k Gamma(n-k) U^-2 V^(k-n) (2U)^-k val_k
  os << "    const R& " << P << "_iV = " << V << "_inv;\n";
  std::string acc, aacc;
  for (int k = 0; k < n && k < int(vals.size()); ++k) {
    if (vals[k].empty()) continue;
    double c = ((n + k) % 2 ? -1.0 : 1.0) * std::tgamma(double(n - k)) * std::pow(4.0, -n) * std::pow(2.0, -k);
    std::string f = "R(" + dstr(c) + ")";
    for (int i = 0; i < n - k; ++i) f += " * " + P + "_iV";
    for (int i = 0; i < 2 + k; ++i) f += " * " + P + "_iU";
    std::string fk = P + "_f" + std::to_string(k);
    os << "    const R " << fk << " = " << f << ";\n";
    acc += (acc.empty() ? "" : " + ") + fk + " * " + vals[k];
    aacc += std::string(aacc.empty() ? "" : " + ") + "fabs(to_double(" + fk + ")) * " + avals[k];
  }
  if (acc.empty()) { acc = "R(0.0)"; aacc = "0.0"; }
  os << "    const R " << out << " = R(" << T.t.sign << ".0) * (" << acc << ");\n";
  os << "    const double " << out << "_abs = " << aacc << ";\n";
  ++st.terms;
}

// One graph's integrand as bytecode: every forest term emitted into one
// function body (polynomials shared across the terms), then compiled.
static qvm::Entry gen_vm_graph(const Graph &g, GenStats &st) {
  auto terms = build_terms(g);
  Emitter E;
  std::vector<std::string> outs;
  for (auto &t : terms) {
    TermInfo T = analyse(g, t);
    std::string o = "term" + std::to_string(outs.size());
    emit_term(E, T, o, st);
    outs.push_back(o);
  }
  std::ostringstream body;
  body << E.os.str() << "    return ";
  for (size_t i = 0; i < outs.size(); ++i) body << (i ? " + " : "") << outs[i];
  body << ";\n";
  qvm::Compiler C(g.n_lines());
  qvm::Entry e;
  e.name = g.name();
  e.n_lines = g.n_lines();
  try {
    e.prog = C.compile(body.str(), outs);
  } catch (const std::exception &x) {
    fprintf(stderr, "qed_gen: %s: %s (graph left out)\n", e.name.c_str(), x.what());
    e.prog.code.clear();
  }
  return e;
}

// All graphs of order n, one per mirror pair (the smaller key; QED_VM_ALL=1:
// both orientations), or the listed ones, on all host threads;
// QED_VM_LIMIT=k keeps the first k.
static int vm_failures = 0;

static void gen_vm_order(const std::string &dir, int n, GenStats &st, const std::vector<int> &only) {
  std::vector<Graph> gs;
  const bool all = getenv("QED_VM_ALL") && atoi(getenv("QED_VM_ALL"));
  const auto every = enumerate_graphs(n);
  if (!only.empty()) {
    for (int i : only) {
      if (i < 0 || size_t(i) >= every.size()) { fprintf(stderr, "qed_gen: graph index %d out of range\n", i); exit(1); }
      gs.push_back(every[size_t(i)]);
    }
  } else {
    for (auto &g : every)
      if (all || !(g.mirror().key() < g.key())) gs.push_back(g);
  }
  if (const char *lim = getenv("QED_VM_LIMIT")) {
    const size_t k = size_t(atol(lim));
    if (k < gs.size()) gs.resize(k);
  }
  std::vector<qvm::Entry> es(gs.size());
  std::vector<GenStats> sts(gs.size());
  // largest graphs (most forest terms) first, so that no long one starts last
  std::vector<size_t> order(gs.size());
  std::vector<size_t> cost(gs.size());
  for (size_t i = 0; i < gs.size(); ++i) { order[i] = i; cost[i] = build_terms(gs[i]).size(); }
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return cost[a] > cost[b]; });
  std::atomic<size_t> next{0};
  unsigned nt = std::max(1u, std::thread::hardware_concurrency());
  if (const char *j = getenv("QED_GEN_JOBS")) nt = std::max(1, atoi(j));
  std::vector<std::thread> th;
  for (unsigned t = 0; t < nt; ++t)
    th.emplace_back([&]() {
      for (size_t k; (k = next.fetch_add(1)) < gs.size();) es[order[k]] = gen_vm_graph(gs[order[k]], sts[order[k]]);
    });
  for (auto &t : th) t.join();
  size_t ins = 0;
  double flops = 0.0;
  int regs = 0;
  for (size_t i = 0; i < es.size(); ++i) {
    st.terms += sts[i].terms;
    st.monos += sts[i].monos;
    ins += es[i].prog.code.size();
    flops += es[i].prog.flops;
    regs = std::max(regs, es[i].prog.n_regs);
  }
  std::vector<qvm::Entry> good;
  size_t kon_max = 0;
  for (auto &e : es)
    if (!e.prog.code.empty()) { good.push_back(e); kon_max = std::max(kon_max, e.prog.kon.size()); }
  if (good.size() != es.size()) vm_failures += int(es.size() - good.size());
  qvm::write_programs(dir + "/vm_n" + std::to_string(n) + ".bin", good);
  fprintf(stderr, "qed_gen: order %d: at most %zu constants in a program\n", n, kon_max);
  fprintf(stderr, "qed_gen: %zu bytecode programs of order %d, %zu instructions, %.0f FP64 ops, at most %d registers\n",
          es.size(), n, ins, flops, regs);
}

int main(int argc, char **argv) {
  if (argc < 3) { fprintf(stderr, "usage: qed_gen out_dir n1 [n2 ...]\n"); return 2; }
  int split_from = 3;
  if (const char *e = getenv("QED_GEN_SPLIT_FROM")) split_from = atoi(e);
  init_gammas();
  init_projectors();
  const std::string dir = argv[1];
  const char *banner =
      "// Generated by qed_gen from the forest-like subtraction formula. Do not edit.\n"
      "// Subtracted Feynman-parametric integrand of one vertex graph, homogeneous\n"
      "// of degree -3n in z; absum receives the sum of the absolute values of all\n"
      "// its monomials (the cancellation measure used by the rounding-error flag;\n"
      "// the magnitudes of the Q coefficients are taken in FP32).\n";
  std::vector<std::string> reg;
  std::vector<int> reg_lines;
  std::vector<long> reg_flops;
  GenStats st;
  for (int ai = 2; ai < argc; ++ai) {
    if (argv[ai][0] == 'v') {
      // bytecode programs for the interpreter kernels: vm_n<n>.bin;
      // "v<n>@<file>": only the graphs whose indices (in the full
      // enumeration) the file lists
      const int n = atoi(argv[ai] + 1);
      std::vector<int> only;
      if (const char *at = strchr(argv[ai], '@')) {
        std::ifstream in(at + 1);
        if (!in) { fprintf(stderr, "qed_gen: cannot read %s\n", at + 1); return 1; }
        for (int x; in >> x;) only.push_back(x);
      }
      gen_vm_order(dir, n, st, only);
      continue;
    }
    int n = atoi(argv[ai]);
    auto gs = enumerate_graphs(n);
    for (size_t gi = 0; gi < gs.size(); ++gi) {
      const Graph &g = gs[gi];
      auto terms = build_terms(g);
      // From loop order `split_from` on, each forest term becomes its own
      // non-inlined device function (compile time grows faster than the
      // size of one straight-line function); below it the terms share one
      // function and its polynomials.
      const bool split = g.n >= split_from;
      Emitter E;
      std::vector<std::string> outs;
      std::ostringstream term_funcs;
      long split_ops = 0;
      for (auto &t : terms) {
        TermInfo T = analyse(g, t);
        std::string o = "term" + std::to_string(outs.size());
        if (!split) {
          emit_term(E, T, o, st);
        } else {
          Emitter Et;
          emit_term(Et, T, "v", st);
          const std::string fn = "qed_t_" + g.name() + "_" + std::to_string(outs.size());
          term_funcs << "template <class R>\n__device__ __noinline__ R " << fn
                     << "(const R* __restrict__ z, double& tabs) {\n" << Et.os.str()
                     << "    tabs = v_abs;\n    return v;\n}\n\n";
          E.os << "    double " << o << "_abs;\n";
          E.os << "    const R " << o << " = " << fn << "<R>(z, " << o << "_abs);\n";
          std::istringstream lines(Et.os.str());
          std::string ln;
          while (std::getline(lines, ln)) {
            if (ln.find("float ") != std::string::npos || ln.find("double ") != std::string::npos ||
                ln.find("_a = ") != std::string::npos || ln.find("_abs") != std::string::npos) continue;
            for (size_t k = 0; k + 2 < ln.size(); ++k)
              if (ln[k] == ' ' && ln[k + 2] == ' ' && (ln[k + 1] == '+' || ln[k + 1] == '-' || ln[k + 1] == '*' || ln[k + 1] == '/')) ++split_ops;
          }
        }
        outs.push_back(o);
      }
      const int id = int(reg.size());
      // algorithmic FP64 operations of the integrand: binary operators in the
      // emitted expressions plus the absum accumulation and the final sum
      {
        // FP64 operations only: the condition-estimate lines (float and
        // double accumulators of absolute values) run on other pipes or are
        // not part of the value
        std::istringstream lines(E.os.str());
        std::string ln;
        long ops = 0;
        while (std::getline(lines, ln)) {
          if (ln.find("float ") != std::string::npos || ln.find("double ") != std::string::npos ||
              ln.find("_a = ") != std::string::npos || ln.find("_abs") != std::string::npos) continue;
          for (size_t k = 0; k + 2 < ln.size(); ++k)
            if (ln[k] == ' ' && ln[k + 2] == ' ' && (ln[k + 1] == '+' || ln[k + 1] == '-' || ln[k + 1] == '*' || ln[k + 1] == '/')) ++ops;
        }
        ops += long(outs.size()) + split_ops;   // the final sum of the terms
        reg_flops.push_back(ops);
      }
      std::ofstream f(dir + "/g_" + std::to_string(id) + ".cuh");
      f << banner << "#pragma once\n\n";
      f << "// " << g.name() << ": " << terms.size() << " forest terms\n";
      f << term_funcs.str();
      f << "template <class R>\n__device__ __forceinline__ R qed_f_" << g.name() << "(const R* __restrict__ z, double& absum) {\n";
      f << E.os.str();
      f << "    absum = 0.0;\n";
      for (auto &o : outs) f << "    absum += " << o << "_abs;\n";
      f << "    return ";
      for (size_t i = 0; i < outs.size(); ++i) f << (i ? " + " : "") << outs[i];
      f << ";\n}\n\n";
      f << "template <int FID> struct qed_gen_f;\n";
      f << "template <> struct qed_gen_f<" << id << "> { template <class R> __device__ static __forceinline__ R eval(const R* __restrict__ z, double& absum) { return qed_f_" << g.name() << "<R>(z, absum); } };\n";
      reg.push_back(g.name());
      reg_lines.push_back(g.n_lines());
    }
  }
  if (reg.empty()) return vm_failures ? 1 : 0;   // bytecode orders only: the registry is the compiled set's
  std::ofstream f(dir + "/qed_registry.h");
  f << "// Generated by qed_gen. Registry of the generated integrands.\n#pragma once\n";
  f << "#define QED_N_GENERATED " << reg.size() << "\n";
  f << "// X(id, lines)\n#define QED_GENERATED_LIST(X)";
  for (size_t i = 0; i < reg.size(); ++i) f << " X(" << i << ", " << reg_lines[i] << ")";
  f << "\n";
  f << "static const double qed_generated_flops[] = {";
  for (size_t i = 0; i < reg.size(); ++i) f << (i ? ", " : "") << reg_flops[i] << ".0";
  f << "};\n";
  f << "static const char* const qed_generated_names[] = {";
  for (size_t i = 0; i < reg.size(); ++i) f << (i ? ", " : "") << "\"" << reg[i] << "\"";
  f << "};\n";
  fprintf(stderr, "qed_gen: %zu graphs, %ld terms, %ld monomials\n", reg.size(), st.terms, st.monos);
  return 0;
}
