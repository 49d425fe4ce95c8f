// qc_qasm.cu -- OpenQASM 2.0 input and output of gate lists (host code).
//
// The paper's library exchanges circuits through openQASM (Sec. 3).  This
// file reads an OpenQASM 2.0 program into qc_gate records and writes gate
// records back.  Register qubits are numbered in declaration order: the
// first qreg's element 0 is qubit 0, the most significant bit of a basis
// index (Definition 1), and so on.
//
// Read: OPENQASM / include (the standard gate library is built in), qreg,
// creg, gate definitions (expanded as macros with their parameters and
// qubit arguments substituted), applications with parameter expressions
// (numbers, pi, + - * / ^, unary minus, sin cos tan exp ln sqrt) and
// register broadcasting (a whole register as an argument applies the gate to
// every element; several whole registers pair up element by element).
// measure and barrier are skipped and counted; reset, if and opaque are
// rejected (QC_ERR_UNSUPPORTED): a state-vector sweep has no classical
// control.
//
// Gates: U, u3, u, u2, u1, p, CX, cx, id, x, y, z, h, s, sdg, t, tdg, sx, sxdg,
// rx, ry, rz, cy, cz, ch, swap, ccx, cswap, crx, cry, crz, cu1, cp, cu3, cu,
// rzz, rxx.  U(t, f, l) = [[cos t/2, -e^{il} sin t/2], [e^{if} sin t/2,
// e^{i(f+l)} cos t/2]] (the OpenQASM 2.0 definition); u2(f, l) = U(pi/2, f, l);
// u1(l) = p(l) = diag(1, e^{il}); cu3 is controlled U without phase, cu(t, f,
// l, g) controlled e^{ig} U; rzz(t) = exp(-i t/2 Z Z), rxx(t) = exp(-i t/2 X X).
#include <cctype>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "qc_common.cuh"

struct qc_program {
  int n = 0;
  int ignored = 0;
  std::vector<qc_gate> gates;
  std::deque<std::vector<double>> mats;     // matrix storage (stable addresses)
};

namespace {

using cd = std::complex<double>;

enum TokKind { T_ID, T_NUM, T_STR, T_SYM, T_END };
struct Tok {
  TokKind k;
  std::string s;
  double v = 0.0;
  int line = 0;
};

struct QasmError {
  int code;
  std::string msg;
};

[[noreturn]] void fail(int code, int line, const std::string& m) {
  throw QasmError{code, "line " + std::to_string(line) + ": " + m};
}

std::vector<Tok> lex(const char* p) {
  std::vector<Tok> out;
  int line = 1;
  while (*p) {
    const char c = *p;
    if (c == '\n') { line++; p++; continue; }
    if (c == ' ' || c == '\t' || c == '\r') { p++; continue; }
    if (c == '/' && p[1] == '/') { while (*p && *p != '\n') p++; continue; }
    if (std::isalpha((unsigned char)c) || c == '_') {
      const char* b = p;
      while (std::isalnum((unsigned char)*p) || *p == '_') p++;
      out.push_back({T_ID, std::string(b, p), 0.0, line});
      continue;
    }
    if (std::isdigit((unsigned char)c) || (c == '.' && std::isdigit((unsigned char)p[1]))) {
      char* e = nullptr;
      const double v = std::strtod(p, &e);
      out.push_back({T_NUM, std::string(p, (const char*)e), v, line});
      p = e;
      continue;
    }
    if (c == '"') {
      const char* b = ++p;
      while (*p && *p != '"' && *p != '\n') p++;
      if (*p != '"') fail(QC_ERR_ARG, line, "unterminated string");
      out.push_back({T_STR, std::string(b, p), 0.0, line});
      p++;
      continue;
    }
    if (c == '-' && p[1] == '>') { out.push_back({T_SYM, "->", 0.0, line}); p += 2; continue; }
    if (c == '=' && p[1] == '=') { out.push_back({T_SYM, "==", 0.0, line}); p += 2; continue; }
    if (std::strchr(";,()[]{}+-*/^", c)) { out.push_back({T_SYM, std::string(1, c), 0.0, line}); p++; continue; }
    fail(QC_ERR_ARG, line, std::string("unexpected character '") + c + "'");
  }
  out.push_back({T_END, "", 0.0, line});
  return out;
}

// A parameter expression, kept as tokens until its variables are known.
struct Expr {
  std::vector<Tok> toks;
};

struct GateDef {
  std::vector<std::string> params, qargs;
  std::vector<Tok> body;                      // tokens between the braces
  int line = 0;
};

class Parser {
 public:
  explicit Parser(std::vector<Tok> t) : t_(std::move(t)) {}

  void program(qc_program& prog) {
    prog_ = &prog;
    while (peek().k != T_END) statement();
    prog.n = nq_;
  }

 private:
  std::vector<Tok> t_;
  size_t i_ = 0;
  qc_program* prog_ = nullptr;
  int nq_ = 0;
  std::map<std::string, std::pair<int, int>> qregs_;   // name -> (first qubit, size)
  std::map<std::string, int> cregs_;
  std::map<std::string, GateDef> defs_;

  const Tok& peek(size_t a = 0) const { return t_[std::min(i_ + a, t_.size() - 1)]; }
  const Tok& next() { return t_[std::min(i_++, t_.size() - 1)]; }
  bool is_sym(const char* s, size_t a = 0) const { return peek(a).k == T_SYM && peek(a).s == s; }
  void expect(const char* s) {
    if (!is_sym(s)) fail(QC_ERR_ARG, peek().line, std::string("expected '") + s + "', found '" + peek().s + "'");
    next();
  }
  std::string ident() {
    if (peek().k != T_ID) fail(QC_ERR_ARG, peek().line, "expected a name, found '" + peek().s + "'");
    return next().s;
  }
  int integer() {
    if (peek().k != T_NUM) fail(QC_ERR_ARG, peek().line, "expected an integer");
    const Tok& k = next();
    if (k.v != std::floor(k.v) || k.v < 0) fail(QC_ERR_ARG, k.line, "expected a non-negative integer");
    return (int)k.v;
  }

  void statement() {
    const Tok& k = peek();
    if (k.k != T_ID) fail(QC_ERR_ARG, k.line, "unexpected '" + k.s + "'");
    const std::string w = k.s;
    if (w == "OPENQASM") {
      next();
      if (peek().k != T_NUM) fail(QC_ERR_ARG, peek().line, "expected a version number");
      if (next().v >= 3.0) fail(QC_ERR_UNSUPPORTED, k.line, "only OpenQASM 2.0 is read");
      expect(";");
    } else if (w == "include") {
      next();
      if (peek().k != T_STR) fail(QC_ERR_ARG, peek().line, "expected a file name");
      next();
      expect(";");
    } else if (w == "qreg" || w == "creg") {
      next();
      const std::string name = ident();
      expect("[");
      const int sz = integer();
      expect("]");
      expect(";");
      if (qregs_.count(name) || cregs_.count(name)) fail(QC_ERR_ARG, k.line, "register '" + name + "' declared twice");
      if (w == "qreg") {
        if (sz < 1 || nq_ + sz > 36) fail(QC_ERR_ARG, k.line, "at most 36 qubits in total");
        qregs_[name] = {nq_, sz};
        nq_ += sz;
      } else {
        cregs_[name] = sz;
      }
    } else if (w == "gate") {
      gate_def();
    } else if (w == "opaque" || w == "reset" || w == "if") {
      fail(QC_ERR_UNSUPPORTED, k.line, "'" + w + "' is not supported (no classical control or opaque gates)");
    } else if (w == "measure" || w == "barrier") {
      next();
      while (!is_sym(";")) {
        if (peek().k == T_END) fail(QC_ERR_ARG, k.line, "missing ';'");
        next();
      }
      next();
      prog_->ignored++;
    } else {
      application();
    }
  }

  void gate_def() {
    const int line = next().line;
    const std::string name = ident();
    GateDef d;
    d.line = line;
    if (is_sym("(")) {
      next();
      if (!is_sym(")")) {
        d.params.push_back(ident());
        while (is_sym(",")) { next(); d.params.push_back(ident()); }
      }
      expect(")");
    }
    d.qargs.push_back(ident());
    while (is_sym(",")) { next(); d.qargs.push_back(ident()); }
    expect("{");
    int depth = 1;
    while (true) {
      if (peek().k == T_END) fail(QC_ERR_ARG, line, "unterminated gate body");
      if (is_sym("{")) depth++;
      if (is_sym("}") && --depth == 0) break;
      d.body.push_back(next());
    }
    next();
    d.body.push_back({T_END, "", 0.0, line});
    defs_[name] = std::move(d);
  }

  // one argument: a register element or a whole register -> list of qubits
  std::vector<int> argument() {
    const int line = peek().line;
    const std::string name = ident();
    auto it = qregs_.find(name);
    if (it == qregs_.end()) fail(QC_ERR_ARG, line, "unknown quantum register '" + name + "'");
    if (is_sym("[")) {
      next();
      const int idx = integer();
      expect("]");
      if (idx >= it->second.second) fail(QC_ERR_ARG, line, name + "[" + std::to_string(idx) + "] is out of range");
      return {it->second.first + idx};
    }
    std::vector<int> v;
    for (int j = 0; j < it->second.second; j++) v.push_back(it->second.first + j);
    return v;
  }

  // parameter expressions as token lists, split at top-level commas
  std::vector<Expr> param_list() {
    std::vector<Expr> out;
    if (!is_sym("(")) return out;
    next();
    if (is_sym(")")) { next(); return out; }
    Expr e;
    int depth = 0;
    while (true) {
      if (peek().k == T_END) fail(QC_ERR_ARG, peek().line, "unterminated parameter list");
      if (is_sym("(")) depth++;
      if (is_sym(")")) {
        if (depth == 0) break;
        depth--;
      }
      if (is_sym(",") && depth == 0) { out.push_back(e); e.toks.clear(); next(); continue; }
      e.toks.push_back(next());
    }
    next();
    out.push_back(e);
    return out;
  }

  void application() {
    const int line = peek().line;
    const std::string name = ident();
    std::vector<Expr> pe = param_list();
    std::vector<double> pv;
    for (const Expr& e : pe) pv.push_back(eval(e, {}, line));
    std::vector<std::vector<int>> args;
    args.push_back(argument());
    while (is_sym(",")) { next(); args.push_back(argument()); }
    expect(";");
    // broadcasting over whole registers
    size_t len = 1;
    for (auto& a : args)
      if (a.size() > 1) {
        if (len > 1 && a.size() != len) fail(QC_ERR_ARG, line, "registers of different sizes in one application");
        len = a.size();
      }
    for (size_t j = 0; j < len; j++) {
      std::vector<int> q;
      for (auto& a : args) q.push_back(a.size() > 1 ? a[j] : a[0]);
      apply(name, pv, q, line, 0);
    }
  }

  // ---- expressions ------------------------------------------------------
  double eval(const Expr& e, const std::map<std::string, double>& vars, int line) {
    std::vector<Tok> toks = e.toks;
    toks.push_back({T_END, "", 0.0, line});
    size_t p = 0;
    const double v = expr(toks, p, vars);
    if (toks[p].k != T_END) fail(QC_ERR_ARG, line, "unexpected '" + toks[p].s + "' in an expression");
    return v;
  }
  double expr(const std::vector<Tok>& t, size_t& p, const std::map<std::string, double>& vars) {
    double v = term(t, p, vars);
    while (t[p].k == T_SYM && (t[p].s == "+" || t[p].s == "-")) {
      const bool add = t[p++].s == "+";
      const double r = term(t, p, vars);
      v = add ? v + r : v - r;
    }
    return v;
  }
  double term(const std::vector<Tok>& t, size_t& p, const std::map<std::string, double>& vars) {
    double v = power(t, p, vars);
    while (t[p].k == T_SYM && (t[p].s == "*" || t[p].s == "/")) {
      const bool mul = t[p++].s == "*";
      const double r = power(t, p, vars);
      v = mul ? v * r : v / r;
    }
    return v;
  }
  double power(const std::vector<Tok>& t, size_t& p, const std::map<std::string, double>& vars) {
    const double b = unary(t, p, vars);
    if (t[p].k == T_SYM && t[p].s == "^") {
      p++;
      return std::pow(b, power(t, p, vars));     // right associative
    }
    return b;
  }
  double unary(const std::vector<Tok>& t, size_t& p, const std::map<std::string, double>& vars) {
    if (t[p].k == T_SYM && t[p].s == "-") { p++; return -unary(t, p, vars); }
    if (t[p].k == T_SYM && t[p].s == "+") { p++; return unary(t, p, vars); }
    return primary(t, p, vars);
  }
  double primary(const std::vector<Tok>& t, size_t& p, const std::map<std::string, double>& vars) {
    const Tok& k = t[p];
    if (k.k == T_NUM) { p++; return k.v; }
    if (k.k == T_SYM && k.s == "(") {
      p++;
      const double v = expr(t, p, vars);
      if (!(t[p].k == T_SYM && t[p].s == ")")) fail(QC_ERR_ARG, k.line, "expected ')'");
      p++;
      return v;
    }
    if (k.k == T_ID) {
      p++;
      if (k.s == "pi") return M_PI;
      auto it = vars.find(k.s);
      if (it != vars.end()) return it->second;
      static const std::map<std::string, double (*)(double)> fns = {
          {"sin", [](double x) { return std::sin(x); }}, {"cos", [](double x) { return std::cos(x); }},
          {"tan", [](double x) { return std::tan(x); }}, {"exp", [](double x) { return std::exp(x); }},
          {"ln", [](double x) { return std::log(x); }},  {"sqrt", [](double x) { return std::sqrt(x); }}};
      auto f = fns.find(k.s);
      if (f != fns.end()) {
        if (!(t[p].k == T_SYM && t[p].s == "(")) fail(QC_ERR_ARG, k.line, "expected '(' after " + k.s);
        p++;
        const double v = expr(t, p, vars);
        if (!(t[p].k == T_SYM && t[p].s == ")")) fail(QC_ERR_ARG, k.line, "expected ')'");
        p++;
        return f->second(v);
      }
      fail(QC_ERR_ARG, k.line, "unknown name '" + k.s + "' in an expression");
    }
    fail(QC_ERR_ARG, k.line, "unexpected '" + k.s + "' in an expression");
  }

  // ---- gates ------------------------------------------------------------
  void need(const std::string& name, const std::vector<double>& pv, const std::vector<int>& q, size_t np, size_t nq,
            int line) {
    if (pv.size() != np || q.size() != nq)
      fail(QC_ERR_ARG, line, "'" + name + "' takes " + std::to_string(np) + " parameters and " + std::to_string(nq) +
                                 " qubits");
    for (size_t a = 0; a < q.size(); a++)
      for (size_t b = a + 1; b < q.size(); b++)
        if (q[a] == q[b]) fail(QC_ERR_ARG, line, "'" + name + "' applied to one qubit twice");
  }

  void named(int kind, const std::vector<int>& tg, const std::vector<int>& ctl, double theta = 0.0) {
    qc_gate g;
    std::memset(&g, 0, sizeof(g));
    g.kind = kind;
    g.nq = (int)tg.size();
    for (size_t j = 0; j < tg.size(); j++) g.qubits[j] = tg[j];
    g.nc = (int)ctl.size();
    for (size_t j = 0; j < ctl.size(); j++) { g.controls[j] = ctl[j]; g.cstates[j] = 1; }
    g.theta = theta;
    prog_->gates.push_back(g);
  }
  void matrix(const std::vector<cd>& U, const std::vector<int>& tg, const std::vector<int>& ctl) {
    std::vector<double> m(2 * U.size());
    for (size_t j = 0; j < U.size(); j++) { m[2 * j] = U[j].real(); m[2 * j + 1] = U[j].imag(); }
    prog_->mats.push_back(std::move(m));
    qc_gate g;
    std::memset(&g, 0, sizeof(g));
    g.kind = QC_GATE_MATRIX;
    g.nq = (int)tg.size();
    for (size_t j = 0; j < tg.size(); j++) g.qubits[j] = tg[j];
    g.nc = (int)ctl.size();
    for (size_t j = 0; j < ctl.size(); j++) { g.controls[j] = ctl[j]; g.cstates[j] = 1; }
    g.matrix = prog_->mats.back().data();
    prog_->gates.push_back(g);
  }
  static std::vector<cd> u3(double t, double f, double l, double gph = 0.0) {
    const cd e = std::exp(cd(0, gph));
    const double c = std::cos(t / 2), s = std::sin(t / 2);
    return {e * c, -e * std::exp(cd(0, l)) * s, e * std::exp(cd(0, f)) * s, e * std::exp(cd(0, f + l)) * c};
  }

  void apply(const std::string& name, const std::vector<double>& pv, const std::vector<int>& q, int line, int depth) {
    if (depth > 64) fail(QC_ERR_ARG, line, "gate definitions nested too deeply");
    auto d = defs_.find(name);
    if (d != defs_.end()) { expand(d->second, name, pv, q, line, depth); return; }
    static const std::map<std::string, int> one = {
        {"x", QC_GATE_X}, {"y", QC_GATE_Y}, {"z", QC_GATE_Z}, {"h", QC_GATE_H}, {"s", QC_GATE_S},
        {"sdg", QC_GATE_SDG}, {"t", QC_GATE_T}, {"tdg", QC_GATE_TDG}};
    static const std::map<std::string, int> rot = {{"rx", QC_GATE_RX}, {"ry", QC_GATE_RY}, {"rz", QC_GATE_RZ},
                                                   {"u1", QC_GATE_P}, {"p", QC_GATE_P}};
    static const std::map<std::string, int> ctl1 = {{"cx", QC_GATE_X}, {"CX", QC_GATE_X}, {"cy", QC_GATE_Y},
                                                    {"cz", QC_GATE_Z}, {"ch", QC_GATE_H}};
    static const std::map<std::string, int> crot = {{"crx", QC_GATE_RX}, {"cry", QC_GATE_RY}, {"crz", QC_GATE_RZ},
                                                    {"cu1", QC_GATE_P}, {"cp", QC_GATE_P}};
    if (one.count(name)) { need(name, pv, q, 0, 1, line); named(one.at(name), {q[0]}, {}); return; }
    if (rot.count(name)) { need(name, pv, q, 1, 1, line); named(rot.at(name), {q[0]}, {}, pv[0]); return; }
    if (ctl1.count(name)) { need(name, pv, q, 0, 2, line); named(ctl1.at(name), {q[1]}, {q[0]}); return; }
    if (crot.count(name)) { need(name, pv, q, 1, 2, line); named(crot.at(name), {q[1]}, {q[0]}, pv[0]); return; }
    if (name == "id" || name == "u0") { need(name, pv, q, name == "u0" ? 1 : 0, 1, line); return; }
    if (name == "U" || name == "u3" || name == "u") {
      need(name, pv, q, 3, 1, line);
      matrix(u3(pv[0], pv[1], pv[2]), {q[0]}, {});
      return;
    }
    if (name == "u2") { need(name, pv, q, 2, 1, line); matrix(u3(M_PI / 2, pv[0], pv[1]), {q[0]}, {}); return; }
    if (name == "sx" || name == "sxdg") {
      need(name, pv, q, 0, 1, line);
      const cd a(0.5, name == "sx" ? 0.5 : -0.5), b(0.5, name == "sx" ? -0.5 : 0.5);
      matrix({a, b, b, a}, {q[0]}, {});
      return;
    }
    if (name == "swap") { need(name, pv, q, 0, 2, line); named(QC_GATE_SWAP, {q[0], q[1]}, {}); return; }
    if (name == "ccx") { need(name, pv, q, 0, 3, line); named(QC_GATE_X, {q[2]}, {q[0], q[1]}); return; }
    if (name == "cswap") { need(name, pv, q, 0, 3, line); named(QC_GATE_SWAP, {q[1], q[2]}, {q[0]}); return; }
    if (name == "cu3") { need(name, pv, q, 3, 2, line); matrix(u3(pv[0], pv[1], pv[2]), {q[1]}, {q[0]}); return; }
    if (name == "cu") { need(name, pv, q, 4, 2, line); matrix(u3(pv[0], pv[1], pv[2], pv[3]), {q[1]}, {q[0]}); return; }
    if (name == "rzz" || name == "rxx") {
      need(name, pv, q, 1, 2, line);
      const double h = pv[0] / 2;
      const cd c(std::cos(h), 0.0), s(0.0, -std::sin(h));
      const cd em = std::exp(cd(0, -h)), ep = std::exp(cd(0, h));
      std::vector<cd> U(16, cd(0));
      if (name == "rzz") {
        U[0] = em; U[5] = ep; U[10] = ep; U[15] = em;
      } else {                                   // cos h I - i sin h X X
        for (int r = 0; r < 4; r++) { U[r * 4 + r] = c; U[r * 4 + (3 - r)] = s; }
      }
      matrix(U, {q[0], q[1]}, {});
      return;
    }
    fail(QC_ERR_ARG, line, "unknown gate '" + name + "'");
  }

  void expand(const GateDef& d, const std::string& name, const std::vector<double>& pv, const std::vector<int>& q,
              int line, int depth) {
    if (pv.size() != d.params.size() || q.size() != d.qargs.size())
      fail(QC_ERR_ARG, line, "'" + name + "' takes " + std::to_string(d.params.size()) + " parameters and " +
                                 std::to_string(d.qargs.size()) + " qubits");
    std::map<std::string, double> vars;
    for (size_t j = 0; j < pv.size(); j++) vars[d.params[j]] = pv[j];
    std::map<std::string, int> qa;
    for (size_t j = 0; j < q.size(); j++) qa[d.qargs[j]] = q[j];
    const std::vector<Tok>& b = d.body;
    size_t p = 0;
    while (b[p].k != T_END) {
      if (b[p].k != T_ID) fail(QC_ERR_ARG, b[p].line, "unexpected '" + b[p].s + "' in the body of " + name);
      const std::string g = b[p].s;
      const int gl = b[p].line;
      p++;
      if (g == "barrier") {
        while (b[p].k != T_END && !(b[p].k == T_SYM && b[p].s == ";")) p++;
        if (b[p].k == T_SYM) p++;
        continue;
      }
      std::vector<double> gv;
      if (b[p].k == T_SYM && b[p].s == "(") {
        p++;
        Expr e;
        int dep = 0;
        while (true) {
          if (b[p].k == T_END) fail(QC_ERR_ARG, gl, "unterminated parameter list");
          if (b[p].k == T_SYM && b[p].s == "(") dep++;
          if (b[p].k == T_SYM && b[p].s == ")") {
            if (dep == 0) break;
            dep--;
          }
          if (b[p].k == T_SYM && b[p].s == "," && dep == 0) { gv.push_back(eval(e, vars, gl)); e.toks.clear(); p++; continue; }
          e.toks.push_back(b[p++]);
        }
        p++;
        if (!e.toks.empty()) gv.push_back(eval(e, vars, gl));
      }
      std::vector<int> gq;
      while (true) {
        if (b[p].k != T_ID || !qa.count(b[p].s)) fail(QC_ERR_ARG, gl, "expected a qubit argument of " + name);
        gq.push_back(qa[b[p].s]);
        p++;
        if (b[p].k == T_SYM && b[p].s == ",") { p++; continue; }
        break;
      }
      if (!(b[p].k == T_SYM && b[p].s == ";")) fail(QC_ERR_ARG, gl, "expected ';' in the body of " + name);
      p++;
      apply(g, gv, gq, gl, depth + 1);
    }
  }
};

// ---- writing --------------------------------------------------------------
struct Writer {
  std::string out;
  void line(const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    out += buf;
    out += "\n";
  }
};

// U = e^{i g} U3(t, f, l)
void zyz(const double* m, double* t, double* f, double* l, double* g) {
  const cd u00(m[0], m[1]), u01(m[2], m[3]), u10(m[4], m[5]), u11(m[6], m[7]);
  *t = 2.0 * std::atan2(std::abs(u10), std::abs(u00));
  if (std::abs(u00) > 1e-14) {
    *g = std::arg(u00);
    if (std::abs(u10) > 1e-14) {
      *f = std::arg(u10) - *g;
      *l = std::arg(-u01) - *g;
    } else {
      *f = 0.0;
      *l = std::arg(u11) - *g;
    }
  } else {
    *l = 0.0;
    *g = std::arg(-u01);
    *f = std::arg(u10) - *g;
  }
}

}  // namespace

extern "C" int qc_qasm_parse(const char* text, qc_program** out) {
  if (!text || !out) return qc_fail(QC_ERR_ARG, "text or out is NULL");
  *out = nullptr;
  auto prog = std::make_unique<qc_program>();
  try {
    Parser p(lex(text));
    p.program(*prog);
  } catch (const QasmError& e) {
    return qc_fail(e.code, "qasm: %s", e.msg.c_str());
  }
  if (prog->n < 1) return qc_fail(QC_ERR_ARG, "qasm: no qreg declared");
  *out = prog.release();
  return QC_OK;
}

extern "C" int qc_program_info(const qc_program* p, int* nqubits, int* ngates, int* nignored) {
  if (!p) return qc_fail(QC_ERR_ARG, "program is NULL");
  if (nqubits) *nqubits = p->n;
  if (ngates) *ngates = (int)p->gates.size();
  if (nignored) *nignored = p->ignored;
  return QC_OK;
}

extern "C" const qc_gate* qc_program_gates(const qc_program* p) {
  return (p && !p->gates.empty()) ? p->gates.data() : nullptr;
}

extern "C" int qc_program_free(qc_program* p) {
  delete p;
  return QC_OK;
}

extern "C" int qc_qasm_write(int n, const qc_gate* gates, int ngates, char* buf, size_t cap, size_t* len) {
  if (n < 1 || n > 36) return qc_fail(QC_ERR_ARG, "n=%d out of range 1..36", n);
  if (ngates < 0 || (ngates > 0 && !gates)) return qc_fail(QC_ERR_ARG, "invalid gate list");
  Writer w;
  w.line("OPENQASM 2.0;");
  w.line("include \"qelib1.inc\";");
  w.line("qreg q[%d];", n);
  static const char* one[] = {nullptr, "h", "x", "y", "z", "s", "sdg", "t", "tdg"};
  for (int i = 0; i < ngates; i++) {
    const qc_gate& g = gates[i];
    if (g.nq < 1 || g.nq > QC_MAX_TARGETS || g.nc < 0 || g.nc > QC_MAX_CONTROLS)
      return qc_fail(QC_ERR_ARG, "gate %d: bad qubit counts", i);
    for (int j = 0; j < g.nq; j++)
      if (g.qubits[j] < 0 || g.qubits[j] >= n) return qc_fail(QC_ERR_ARG, "gate %d: qubit out of range", i);
    for (int j = 0; j < g.nc; j++) {
      if (g.controls[j] < 0 || g.controls[j] >= n) return qc_fail(QC_ERR_ARG, "gate %d: control out of range", i);
      if (g.cstates[j] != 0 && g.cstates[j] != 1) return qc_fail(QC_ERR_ARG, "gate %d: control state", i);
    }
    // controls in state 0: conjugate with X
    for (int j = 0; j < g.nc; j++)
      if (g.cstates[j] == 0) w.line("x q[%d];", g.controls[j]);
    const int c0 = g.nc > 0 ? g.controls[0] : -1;
    const int t0 = g.qubits[0];
    bool ok = true;
    if (g.kind >= QC_GATE_H && g.kind <= QC_GATE_TDG && g.nq == 1) {
      if (g.nc == 0) w.line("%s q[%d];", one[g.kind], t0);
      else if (g.nc == 1 && (g.kind == QC_GATE_X || g.kind == QC_GATE_Y || g.kind == QC_GATE_Z || g.kind == QC_GATE_H))
        w.line("c%s q[%d],q[%d];", one[g.kind], c0, t0);
      else if (g.nc == 2 && g.kind == QC_GATE_X) w.line("ccx q[%d],q[%d],q[%d];", g.controls[0], g.controls[1], t0);
      else ok = false;
    } else if ((g.kind == QC_GATE_P || g.kind == QC_GATE_RX || g.kind == QC_GATE_RY || g.kind == QC_GATE_RZ) && g.nq == 1) {
      const char* nm = g.kind == QC_GATE_P ? "u1" : g.kind == QC_GATE_RX ? "rx" : g.kind == QC_GATE_RY ? "ry" : "rz";
      if (g.nc == 0) w.line("%s(%.17g) q[%d];", nm, g.theta, t0);
      else if (g.nc == 1) w.line("c%s(%.17g) q[%d],q[%d];", nm, g.theta, c0, t0);
      else ok = false;
    } else if (g.kind == QC_GATE_SWAP && g.nq == 2) {
      if (g.nc == 0) w.line("swap q[%d],q[%d];", g.qubits[0], g.qubits[1]);
      else if (g.nc == 1) w.line("cswap q[%d],q[%d],q[%d];", c0, g.qubits[0], g.qubits[1]);
      else ok = false;
    } else if (g.kind == QC_GATE_MATRIX && g.nq == 1 && g.matrix && g.nc <= 1) {
      double t, f, l, gp;
      zyz(g.matrix, &t, &f, &l, &gp);
      if (g.nc == 0) {
        w.line("u3(%.17g,%.17g,%.17g) q[%d];", t, f, l, t0);   // global phase e^{i g} dropped
      } else {
        w.line("cu3(%.17g,%.17g,%.17g) q[%d],q[%d];", t, f, l, c0, t0);
        w.line("u1(%.17g) q[%d];", gp, c0);                    // the phase on the control's 1 half
      }
    } else {
      ok = false;
    }
    if (!ok)
      return qc_fail(QC_ERR_UNSUPPORTED, "gate %d has no OpenQASM 2.0 form here (kind %d, %d targets, %d controls)",
                     i, g.kind, g.nq, g.nc);
    for (int j = 0; j < g.nc; j++)
      if (g.cstates[j] == 0) w.line("x q[%d];", g.controls[j]);
  }
  if (len) *len = w.out.size();
  if (buf && cap > 0) {
    if (cap <= w.out.size()) return qc_fail(QC_ERR_ARG, "buffer of %zu bytes, %zu needed", cap, w.out.size() + 1);
    std::memcpy(buf, w.out.c_str(), w.out.size() + 1);
  }
  return QC_OK;
}
