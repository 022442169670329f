// Bytecode back end of the integrand generator (host C++, build time).
//
// From four loops on, a graph's subtracted integrand is tens to hundreds of
// thousands of FP64 operations (Sec. 3 of the paper reports 500 GB of
// compiled code for the 5-loop set); compiling one straight-line function
// per graph no longer fits a build.  Instead the generated function text
// (the same text the compiled path uses, with polynomials shared across the
// graph's forest terms) is parsed and translated into a program for a small
// accumulator machine that one generic CUDA kernel interprets.
//
// Machine (qed_vm.cuh is the device side):
//   per thread: an accumulator (v: value, e: FP32 absolute-value lane), a
//   register file R[0..n_regs) of (v, e) pairs (z[0..N) preloaded in
//   R[0..N) with e = z), and a double W that collects the monomial
//   absolute sum of the integrand;
//   per program: a table K of constants (operand flag 4096 selects K, with
//   e = |K|).
//   The e lane follows the value lane through +, *, fma with the operands'
//   e values; for the quantities whose magnitude the compiled path takes as
//   |value| (the graph polynomials, 1 +- A, C, K, B_ij, 1/U, 1/V and the
//   prefactors) ABS sets e = |v|.  This makes e of every Horner-form sum the
//   sum of the absolute values of its monomials, exactly what the compiled
//   path accumulates; W receives |prefactor| * e(block value) per forest term
//   in double, as the compiled path does.
//
// The code generator works on micro-operations:
//   END                          v, W are the integrand and its absolute sum
//   LD a        acc = a
//   ADD a       acc = acc + a
//   MUL a       acc = acc * a
//   FMA a b     acc = acc * a + b
//   FMAC a b    acc = a * b + acc
//   RCP         acc = 1 / acc          (e = |acc|)
//   ABS         e = |v|
//   ST a        R[a] = acc
//   ACCW a b    W += |a.v| * b.e
//   LDMUL a b   acc = a * b
// (operands: a register index, or 4096 + a constant index), and fuses them
// into 64-bit instructions that the interpreter executes without a dispatch
// on the operation:
//   lo = A | B << 13,  hi = XA | ZO << 1 | SPEC << 2 | NOCOMP << 5 | D << 6
//   1. unless NOCOMP:  X = XA ? A : acc,  O = XA ? acc : A,
//                      acc = X * B + (ZO ? O : 0)           (e lane alike)
//   2. SPEC 1 RCP: acc = 1 / acc, e = |acc|;  2 ABS: e = |acc|;
//      3 ACCW: W += |A.v| * B.e;  4 END
//   3. D != 0: R[D] = acc                     (register 0 is z[0], never stored)
// LD a = (XA, A = a, B = 1); ADD a = (A = a, B = 1, ZO); MUL a = (B = a);
// FMA a b = (A = b, B = a, ZO); FMAC a b = (XA, A = a, B = b, ZO);
// LDMUL a b = (XA, A = a, B = b).  Each value is bit-identical to the
// micro-operation's (x * 1 + 0 and x * y + 0 round like x and x * y).
// The interpreter reads an instruction's operands before the previous
// instruction stores, so no instruction reads the register the one before
// it writes: where that would happen a no-operation (NOCOMP, constant
// operands, no store) is put between them.
#pragma once
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <set>
#include <stdexcept>
#include <sstream>
#include <string>
#include <vector>

namespace qvm {

enum Op : uint32_t { END = 0, LD, ADD, MUL, FMA, FMAC, RCP, ABS, ST, ACCW, LDMUL };
constexpr int KFLAG = 4096;         // operand >= KFLAG: constant K[operand - KFLAG]
constexpr int MAX_REGS = 1023;
constexpr int MAX_KON = 4096;

// micro-operation word: op[0:4) a[4:17) b[17:30)
inline uint32_t enc(Op op, int a = 0, int b = 0) {
  return uint32_t(op) | (uint32_t(a) << 4) | (uint32_t(b) << 17);
}

enum : uint32_t { SP_NONE = 0, SP_RCP = 1, SP_ABS = 2, SP_ACCW = 3, SP_END = 4 };
constexpr uint32_t NOCOMP = 32u;

inline uint64_t word(int A, int B, int D, bool xa, bool zo, uint32_t spec, bool nocomp) {
  const uint32_t lo = uint32_t(A) | (uint32_t(B) << 13);
  const uint32_t hi = uint32_t(xa) | (uint32_t(zo) << 1) | (spec << 2) | (nocomp ? NOCOMP : 0u) | (uint32_t(D) << 6);
  return uint64_t(lo) | (uint64_t(hi) << 32);
}

// ---------------------------------------------------------------------------
// expression trees of the emitted text
// ---------------------------------------------------------------------------
struct Ex {
  enum K { Z, VAR, CON, ADDN, MULN, INV } k;
  int idx = 0;          // Z: line index
  double c = 0.0;       // CON
  std::string name;     // VAR
  std::vector<Ex> ch;
  bool leaf() const { return k == Z || k == VAR || k == CON; }
};

struct Parser {
  const std::string s;
  size_t p = 0;
  explicit Parser(const std::string &str) : s(str) {}
  void ws() { while (p < s.size() && s[p] == ' ') ++p; }
  [[noreturn]] void fail(const char *what) {
    fprintf(stderr, "vm parser: %s at '%s'\n", what, s.substr(p, 60).c_str());
    exit(1);
  }
  bool eat(const char *t) {
    ws();
    const size_t n = strlen(t);
    if (s.compare(p, n, t) == 0) { p += n; return true; }
    return false;
  }
  std::string ident() {
    ws();
    size_t q = p;
    while (q < s.size() && (isalnum((unsigned char)s[q]) || s[q] == '_')) ++q;
    if (q == p) fail("identifier expected");
    std::string r = s.substr(p, q - p);
    p = q;
    return r;
  }
  Ex atom() {
    ws();
    if (eat("R(")) {
      char *end = nullptr;
      Ex e; e.k = Ex::CON; e.c = strtod(s.c_str() + p, &end);
      p = size_t(end - s.c_str());
      if (!eat(")")) fail("')' after constant");
      return e;
    }
    if (eat("z[")) {
      Ex e; e.k = Ex::Z; e.idx = int(strtol(s.c_str() + p, nullptr, 10));
      while (p < s.size() && isdigit((unsigned char)s[p])) ++p;
      if (!eat("]")) fail("']'");
      return e;
    }
    if (eat("(")) {
      Ex e = sum();
      if (!eat(")")) fail("')'");
      return e;
    }
    Ex e; e.k = Ex::VAR; e.name = ident();
    return e;
  }
  Ex prod() {
    Ex first = atom();
    std::vector<Ex> fs;
    fs.push_back(first);
    for (;;) {
      if (eat("*")) { fs.push_back(atom()); continue; }
      if (eat("/")) {
        Ex den = atom();
        Ex num = fs.back();
        fs.pop_back();
        if (num.k != Ex::CON || num.c != 1.0) fail("only 1 / x is generated");
        Ex inv; inv.k = Ex::INV; inv.ch.push_back(den);
        fs.push_back(inv);
        continue;
      }
      break;
    }
    if (fs.size() == 1) return fs[0];
    Ex m; m.k = Ex::MULN;
    for (auto &f : fs) {
      if (f.k == Ex::MULN) for (auto &g : f.ch) m.ch.push_back(g);
      else m.ch.push_back(f);
    }
    return m;
  }
  Ex sum() {
    std::vector<Ex> ts;
    ts.push_back(prod());
    while (eat("+")) ts.push_back(prod());
    if (ts.size() == 1) return ts[0];
    Ex a; a.k = Ex::ADDN;
    for (auto &t : ts) {
      if (t.k == Ex::ADDN) for (auto &g : t.ch) a.ch.push_back(g);
      else a.ch.push_back(t);
    }
    return a;
  }
};

// ---------------------------------------------------------------------------
// statements
// ---------------------------------------------------------------------------
struct Stmt {
  enum K { DEF, UPD, TERM, RET } k;
  std::string lhs;
  Ex rhs;
};

struct Program {
  std::vector<uint32_t> ins;      // micro-operations
  std::vector<uint64_t> code;     // fused instructions (what the file holds)
  std::vector<double> kon;
  int n_regs = 0;
  double flops = 0.0;
};

static void collect_uses(const Ex &e, std::vector<std::string> &out) {
  if (e.k == Ex::VAR) out.push_back(e.name);
  for (auto &c : e.ch) collect_uses(c, out);
}

static void find_abs_marks(const std::string &ln, std::set<std::string> &abs_names) {
  for (const char *pat : {"to_double("}) {
    size_t q = 0;
    while ((q = ln.find(pat, q)) != std::string::npos) {
      q += strlen(pat);
      size_t r = q;
      while (r < ln.size() && (isalnum((unsigned char)ln[r]) || ln[r] == '_')) ++r;
      if (r < ln.size() && ln[r] == ')') abs_names.insert(ln.substr(q, r - q));
    }
  }
}

class Compiler {
 public:
  Compiler(int n_lines) : N(n_lines) {
    for (int i = 0; i < MAX_REGS; ++i) used[i] = false;
    for (int i = 0; i < N; ++i) used[i] = true;      // z
    hi = N;
  }

  // body: the statements of one graph's integrand function; terms: the
  // names of the forest-term outputs in summation order
  Program compile(const std::string &body, const std::vector<std::string> &terms) {
    parse(body, terms);
    // drop values nothing uses (e.g. a line's C or K polynomial that no
    // monomial needs): backward pass from the terms and the return
    {
      std::set<std::string> live;
      std::vector<Stmt> kept;
      for (size_t j = st.size(); j-- > 0;) {
        const Stmt &S = st[j];
        const bool keep = S.k == Stmt::TERM || S.k == Stmt::RET || live.count(S.lhs);
        if (!keep) continue;
        if (S.k == Stmt::DEF) live.erase(S.lhs);
        std::vector<std::string> u;
        collect_uses(S.rhs, u);
        for (auto &n : u) live.insert(n);
        kept.push_back(S);
      }
      st.assign(kept.rbegin(), kept.rend());
    }
    // last use of every name (alias-resolved)
    std::map<std::string, size_t> last;
    for (size_t i = 0; i < st.size(); ++i) {
      if (st[i].k == Stmt::RET) continue;
      std::vector<std::string> u;
      collect_uses(st[i].rhs, u);
      for (auto &n : u) last[n] = i;
      if (st[i].k == Stmt::UPD) last[st[i].lhs] = std::max(last[st[i].lhs], i);
    }
    int freg = -1;                   // running sum of the forest terms
    for (size_t i = 0; i < st.size(); ++i) {
      const Stmt &S = st[i];
      if (S.k == Stmt::RET) {
        // the return statement sums the terms in order: freg holds that sum
        if (freg < 0) emit(LD, kon(0.0)); else emit(LD, freg);
        emit(END);
        break;
      }
      if (S.k == Stmt::TERM) {
        gen_term(S.rhs);
        if (freg < 0) freg = alloc(); else emit(ADD, freg);
        emit(ST, freg);
        std::vector<std::string> u;
        collect_uses(S.rhs, u);
        for (auto &n : u) if (last[n] == i) release(n);
        continue;
      }
      gen(S.rhs);
      // operands whose last use is this statement are free now (acc holds
      // the result)
      std::vector<std::string> u;
      collect_uses(S.rhs, u);
      for (auto &n : u) if (last[n] == i && n != S.lhs) release(n);
      if (S.k == Stmt::DEF) {
        if (abs_names.count(S.lhs)) emit(ABS);
        if (!last.count(S.lhs)) continue;                 // value never used
        const int r = alloc();
        reg[S.lhs] = r;
        emit(ST, r);
      } else {                                            // UPD: same register
        if (abs_names.count(S.lhs)) emit(ABS);
        emit(ST, reg.at(S.lhs));
        if (last[S.lhs] == i) release(S.lhs);
      }
    }
    P.n_regs = hi;
    fuse();
    return P;
  }

 private:
  int N;
  bool used[MAX_REGS];
  int hi;
  std::vector<Stmt> st;
  std::map<std::string, std::string> alias;
  std::set<std::string> abs_names, abs_lane;
  std::map<std::string, int> reg;
  std::map<double, int> kidx;
  Program P;

  std::string resolve(const std::string &n) const {
    auto it = alias.find(n);
    return it == alias.end() ? n : resolve(it->second);
  }
  void resolve_all(Ex &e) {
    if (e.k == Ex::VAR) e.name = resolve(e.name);
    for (auto &c : e.ch) resolve_all(c);
  }

  void parse(const std::string &body, const std::vector<std::string> &terms) {
    parse_lines(body, terms);
    std::set<std::string> r;
    for (auto &n : abs_names) r.insert(resolve(n));
    abs_names.swap(r);
  }
  void parse_lines(const std::string &body, const std::vector<std::string> &terms) {
    std::set<std::string> termset(terms.begin(), terms.end());
    std::istringstream in(body);
    std::string ln;
    while (std::getline(in, ln)) {
      size_t a = ln.find_first_not_of(' ');
      if (a == std::string::npos) continue;
      std::string t = ln.substr(a);
      if (!t.empty() && t.back() == ';') t.pop_back();
      find_abs_marks(t, abs_names);
      auto starts = [&](const char *pre) { return t.compare(0, strlen(pre), pre) == 0; };
      if (starts("const float ") || starts("const double ") || starts("double ")) {
        // absolute-value lane declarations: remember their names
        size_t q = t.find(' ', starts("double ") ? 0 : 6) + 1;
        size_t r = t.find_first_of(" ;=", q);
        abs_lane.insert(t.substr(q, r - q));
        continue;
      }
      if (starts("absum")) continue;
      if (starts("const R& ")) {
        size_t eq = t.find(" = ");
        std::string l = t.substr(9, eq - 9), r = t.substr(eq + 3);
        alias[l] = r;
        continue;
      }
      if (starts("return ")) {
        Stmt S; S.k = Stmt::RET;
        Parser pp(t.substr(7)); S.rhs = pp.sum();
        resolve_all(S.rhs);
        st.push_back(S);
        continue;
      }
      Stmt S;
      std::string rest;
      if (starts("const R ")) { S.k = Stmt::DEF; rest = t.substr(8); }
      else if (starts("R ")) { S.k = Stmt::DEF; rest = t.substr(2); }
      else { S.k = Stmt::UPD; rest = t; }
      size_t eq = rest.find(" = ");
      if (eq == std::string::npos) { fprintf(stderr, "vm: unparsed line '%s'\n", t.c_str()); exit(1); }
      S.lhs = rest.substr(0, eq);
      if (S.k == Stmt::UPD && abs_lane.count(S.lhs)) continue;
      std::string rhs = rest.substr(eq + 3);
      if (S.k == Stmt::UPD) {
        // name = name + EXPR: keep EXPR, accumulate into the same register
        const std::string pre = S.lhs + " + ";
        if (rhs.compare(0, pre.size(), pre) != 0) { fprintf(stderr, "vm: bad update '%s'\n", t.c_str()); exit(1); }
      }
      if (termset.count(S.lhs)) S.k = Stmt::TERM;
      Parser pp(rhs);
      S.rhs = pp.sum();
      if (pp.p != rhs.size()) { pp.ws(); if (pp.p != rhs.size()) pp.fail("trailing text"); }
      resolve_all(S.rhs);
      st.push_back(S);
    }
  }

  int alloc() {
    for (int r = N; r < MAX_REGS; ++r)
      if (!used[r]) { used[r] = true; if (r + 1 > hi) hi = r + 1; return r; }
    throw std::runtime_error("out of registers");
  }
  void free_reg(int r) { if (r >= N) used[r] = false; }
  void release(const std::string &n) {
    auto it = reg.find(n);
    if (it == reg.end()) return;
    free_reg(it->second);
    reg.erase(it);
  }
  // micro-operations -> fused instructions: a compute step, then an optional
  // special (RCP / ABS), then an optional store, share one instruction
  void fuse() {
    const int one = kon(1.0), zero = kon(0.0);
    auto &C = P.code;
    C.clear();
    bool open = false;          // last instruction can still take a special / store
    bool has_spec = false, has_st = false;
    for (uint32_t w : P.ins) {
      const int op = int(w & 15u), a = int((w >> 4) & 8191u), b = int((w >> 17) & 8191u);
      auto put = [&](uint64_t x, bool can_extend) {
        C.push_back(x);
        open = can_extend;
        has_spec = false;
        has_st = false;
      };
      switch (op) {
        case LD: put(word(a, one, 0, true, false, SP_NONE, false), true); break;
        case ADD: put(word(a, one, 0, false, true, SP_NONE, false), true); break;
        case MUL: put(word(zero, a, 0, false, false, SP_NONE, false), true); break;
        case FMA: put(word(b, a, 0, false, true, SP_NONE, false), true); break;
        case FMAC: put(word(a, b, 0, true, true, SP_NONE, false), true); break;
        case LDMUL: put(word(a, b, 0, true, false, SP_NONE, false), true); break;
        case RCP:
        case ABS: {
          const uint32_t sp = op == RCP ? SP_RCP : SP_ABS;
          if (open && !has_spec && !has_st) { C.back() |= uint64_t(sp) << 34; has_spec = true; }
          else { put(word(zero, one, 0, false, false, sp, true), true); has_spec = true; }
          break;
        }
        case ST:
          if (open && !has_st) { C.back() |= uint64_t(uint32_t(a)) << (32 + 6); has_st = true; }
          else { put(word(zero, one, a, false, false, SP_NONE, true), false); }
          break;
        case ACCW: put(word(a, b, 0, false, false, SP_ACCW, true), false); break;
        case END: put(word(zero, one, 0, false, false, SP_END, true), false); break;
        default: fprintf(stderr, "vm: bad micro-operation\n"); exit(1);
      }
    }
    // separate read-after-write neighbours
    std::vector<uint64_t> out;
    out.reserve(C.size() + C.size() / 8);
    for (size_t i = 0; i < C.size(); ++i) {
      if (i > 0) {
        const uint32_t d = uint32_t(C[i - 1] >> (32 + 6)) & 1023u;
        const uint32_t a = uint32_t(C[i]) & 8191u, b = uint32_t(C[i] >> 13) & 8191u;
        if (d != 0 && (a == d || b == d)) out.push_back(word(zero, one, 0, false, false, SP_NONE, true));
      }
      out.push_back(C[i]);
    }
    C.swap(out);
  }

  int kon(double c) {
    auto it = kidx.find(c);
    if (it != kidx.end()) return KFLAG + it->second;
    if (int(P.kon.size()) >= MAX_KON) throw std::runtime_error("more than 4096 constants");
    kidx[c] = int(P.kon.size());
    P.kon.push_back(c);
    return KFLAG + int(P.kon.size()) - 1;
  }
  int opnd(const Ex &e) {
    if (e.k == Ex::Z) return e.idx;
    if (e.k == Ex::CON) return kon(e.c);
    auto it = reg.find(e.name);
    if (it == reg.end()) { fprintf(stderr, "vm: %s used before definition\n", e.name.c_str()); exit(1); }
    return it->second;
  }
  void emit(Op op, int a = 0, int b = 0) {
    P.ins.push_back(enc(op, a, b));
    switch (op) {
      case ADD: case MUL: case RCP: case LDMUL: P.flops += 1.0; break;
      case FMA: case FMAC: P.flops += 2.0; break;
      default: break;
    }
  }

  // acc = value of e
  void gen(const Ex &e) {
    switch (e.k) {
      case Ex::Z: case Ex::VAR: case Ex::CON: emit(LD, opnd(e)); return;
      case Ex::INV: gen(e.ch[0]); emit(RCP); return;
      case Ex::MULN: gen_mul(e.ch); return;
      case Ex::ADDN: gen_add(e.ch); return;
    }
  }
  void gen_mul(const std::vector<Ex> &fs) {
    std::vector<const Ex *> lv, cx;
    for (auto &f : fs) (f.leaf() ? lv : cx).push_back(&f);
    std::vector<int> tmps;
    size_t li = 0;
    if (cx.empty()) {
      if (lv.size() >= 2) { emit(LDMUL, opnd(*lv[0]), opnd(*lv[1])); li = 2; }
      else { emit(LD, opnd(*lv[0])); li = 1; }
    } else {
      for (size_t i = 0; i + 1 < cx.size(); ++i) {
        gen(*cx[i]);
        const int t = alloc();
        emit(ST, t);
        tmps.push_back(t);
      }
      gen(*cx.back());
    }
    for (; li < lv.size(); ++li) emit(MUL, opnd(*lv[li]));
    for (int t : tmps) { emit(MUL, t); free_reg(t); }
  }
  void gen_add(const std::vector<Ex> &ts) {
    std::vector<const Ex *> simple, fma, cx;
    for (auto &t : ts) {
      if (t.leaf()) simple.push_back(&t);
      else if (t.k == Ex::MULN) {
        int nl = 0;
        for (auto &f : t.ch) nl += f.leaf();
        if (nl == int(t.ch.size()) && nl == 2) simple.push_back(&t);
        else if (nl >= 1 && nl == int(t.ch.size()) - 1) fma.push_back(&t);
        else cx.push_back(&t);
      } else cx.push_back(&t);
    }
    bool started = false;
    for (const Ex *c : cx) {
      if (!started) { gen(*c); started = true; continue; }
      const int t = alloc();
      emit(ST, t);
      gen(*c);
      emit(ADD, t);
      free_reg(t);
    }
    size_t f0 = 0;
    if (!started && !fma.empty()) {
      int ad = -1;
      for (size_t i = 0; i < simple.size(); ++i) if (simple[i]->leaf()) { ad = int(i); break; }
      const Ex *x = nullptr;
      std::vector<const Ex *> ls;
      for (auto &c : fma[0]->ch) { if (c.leaf()) ls.push_back(&c); else x = &c; }
      gen(*x);
      for (size_t i = 0; i + 1 < ls.size(); ++i) emit(MUL, opnd(*ls[i]));
      if (ad >= 0) { emit(FMA, opnd(*ls.back()), opnd(*simple[ad])); simple.erase(simple.begin() + ad); }
      else emit(MUL, opnd(*ls.back()));
      started = true;
      f0 = 1;
    }
    for (const Ex *s : simple) {
      if (s->leaf()) emit(started ? ADD : LD, opnd(*s));
      else emit(started ? FMAC : LDMUL, opnd(s->ch[0]), opnd(s->ch[1]));
      started = true;
    }
    for (size_t fi = f0; fi < fma.size(); ++fi) {
      const Ex *f = fma[fi];
      const Ex *x = nullptr;
      std::vector<const Ex *> ls;
      for (auto &c : f->ch) { if (c.leaf()) ls.push_back(&c); else x = &c; }
      if (!started) {
        gen(*x);
        for (auto *l : ls) emit(MUL, opnd(*l));
        started = true;
        continue;
      }
      const int t = alloc();
      emit(ST, t);
      gen(*x);
      for (size_t i = 0; i + 1 < ls.size(); ++i) emit(MUL, opnd(*ls[i]));
      emit(FMA, opnd(*ls.back()), t);
      free_reg(t);
    }
  }
  // term = s * (f_0 * X_0 + f_1 * X_1 + ...): the value, and W += |f_k| e(X_k)
  void gen_term(const Ex &e) {
    if (e.k != Ex::MULN || e.ch.size() < 2 || e.ch[0].k != Ex::CON) { fprintf(stderr, "vm: bad term form\n"); exit(1); }
    const double s = e.ch[0].c;
    std::vector<Ex> parts;
    if (e.ch.size() == 2 && e.ch[1].k == Ex::CON && e.ch[1].c == 0.0) { emit(LD, kon(0.0)); return; }
    if (e.ch.size() == 3) { Ex m; m.k = Ex::MULN; m.ch = {e.ch[1], e.ch[2]}; parts.push_back(m); }
    else if (e.ch[1].k == Ex::ADDN) parts = e.ch[1].ch;
    else parts.push_back(e.ch[1]);
    std::vector<std::pair<int, int>> fx;          // (f register, X register)
    std::vector<int> tmps;
    for (auto &pt : parts) {
      if (pt.k != Ex::MULN || pt.ch.size() != 2 || pt.ch[0].k != Ex::VAR) { fprintf(stderr, "vm: bad term part\n"); exit(1); }
      const int f = opnd(pt.ch[0]);
      int x;
      if (pt.ch[1].leaf()) x = opnd(pt.ch[1]);
      else { gen(pt.ch[1]); x = alloc(); emit(ST, x); tmps.push_back(x); }
      fx.push_back({f, x});
    }
    for (auto &p : fx) emit(ACCW, p.first, p.second);
    for (size_t i = 0; i < fx.size(); ++i) emit(i ? FMAC : LDMUL, fx[i].first, fx[i].second);
    if (s != 1.0) emit(MUL, kon(s));
    for (int t : tmps) free_reg(t);
  }
};

// ---------------------------------------------------------------------------
// program file
// ---------------------------------------------------------------------------
// Layout (little endian): "QEDVM004", u32 count, u32 0, then per program a
// 64-byte name, i32 n_lines, n_regs, n_ins, n_kon, f64 flops, the n_ins
// 64-bit instructions and the constants.
struct Entry {
  std::string name;
  int n_lines;
  Program prog;
};

inline void write_programs(const std::string &path, const std::vector<Entry> &es) {
  FILE *f = fopen(path.c_str(), "wb");
  if (!f) { fprintf(stderr, "vm: cannot write %s\n", path.c_str()); exit(1); }
  fwrite("QEDVM004", 1, 8, f);
  const uint32_t hdr[2] = {uint32_t(es.size()), 0u};
  fwrite(hdr, 4, 2, f);
  for (auto &e : es) {
    char nm[64] = {0};
    strncpy(nm, e.name.c_str(), 63);
    fwrite(nm, 1, 64, f);
    const int32_t m[4] = {e.n_lines, e.prog.n_regs, int32_t(e.prog.code.size()), int32_t(e.prog.kon.size())};
    fwrite(m, 4, 4, f);
    fwrite(&e.prog.flops, 8, 1, f);
    fwrite(e.prog.code.data(), 8, e.prog.code.size(), f);
    fwrite(e.prog.kon.data(), 8, e.prog.kon.size(), f);
  }
  fclose(f);
}

}  // namespace qvm
