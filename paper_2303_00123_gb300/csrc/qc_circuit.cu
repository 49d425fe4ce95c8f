// qc_circuit.cu -- circuit driver: named gates, greedy gate fusion, timing,
// CUDA-graph capture.
//
// A circuit is applied gate by gate, each gate being one sweep over the
// state (QCLAB++ Sec. 3 applies the circuit's gates in order; Sec. 4 notes
// that the GPU time then scales with the number of gates).  With fuse_k >= 2
// runs of gates are first merged on the host into dense k-qubit blocks, so
// that one sweep applies many gates.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "qc_common.cuh"

namespace {

using cd = std::complex<double>;

// Matrix of a named gate (host, FP64).  P(theta) = diag(1, e^{i theta});
// RX/RY/RZ(theta) = exp(-i theta P / 2) (the rotation gates of Fig. 5).
int named_matrix(const qc_gate& g, std::vector<cd>& U) {
  const double r2 = 1.0 / std::sqrt(2.0);
  const double t = g.theta;
  const cd I(0, 1);
  switch (g.kind) {
    case QC_GATE_H: U = {r2, r2, r2, -r2}; return 1;
    case QC_GATE_X: U = {0, 1, 1, 0}; return 1;
    case QC_GATE_Y: U = {0, -I, I, 0}; return 1;
    case QC_GATE_Z: U = {1, 0, 0, -1}; return 1;
    case QC_GATE_S: U = {1, 0, 0, I}; return 1;
    case QC_GATE_SDG: U = {1, 0, 0, -I}; return 1;
    case QC_GATE_T: U = {1, 0, 0, std::polar(1.0, M_PI / 4)}; return 1;
    case QC_GATE_TDG: U = {1, 0, 0, std::polar(1.0, -M_PI / 4)}; return 1;
    case QC_GATE_P: U = {1, 0, 0, std::polar(1.0, t)}; return 1;
    case QC_GATE_RX: U = {std::cos(t / 2), -I * std::sin(t / 2), -I * std::sin(t / 2), std::cos(t / 2)}; return 1;
    case QC_GATE_RY: U = {std::cos(t / 2), -std::sin(t / 2), std::sin(t / 2), std::cos(t / 2)}; return 1;
    case QC_GATE_RZ: U = {std::polar(1.0, -t / 2), 0, 0, std::polar(1.0, t / 2)}; return 1;
    case QC_GATE_SWAP: U.assign(16, 0); U[0] = U[6] = U[9] = U[15] = 1; return 2;
    default: return 0;
  }
}

// Resolve a gate record into (targets, controls, matrix) and validate it.
struct Resolved {
  int k, nc;
  int t[QC_MAX_TARGETS], c[QC_MAX_CONTROLS], cs[QC_MAX_CONTROLS];
  std::vector<cd> U;
};

int resolve(int n, const qc_gate& g, Resolved& R) {
  int k;
  if (g.kind == QC_GATE_MATRIX) {
    k = g.nq;
    if (k < 1 || k > QC_MAX_TARGETS) return qc_fail(QC_ERR_ARG, "matrix gate with nq=%d", g.nq);
    if (!g.matrix) return qc_fail(QC_ERR_ARG, "matrix gate without a matrix");
    const int D = 1 << k;
    R.U.resize((size_t)D * D);
    for (int i = 0; i < D * D; i++) R.U[i] = cd(g.matrix[2 * i], g.matrix[2 * i + 1]);
  } else {
    k = named_matrix(g, R.U);
    if (k == 0) return qc_fail(QC_ERR_ARG, "unknown gate kind %d", g.kind);
    if (g.nq != k) return qc_fail(QC_ERR_ARG, "gate kind %d acts on %d qubit(s), nq=%d", g.kind, k, g.nq);
  }
  if (g.nc < 0 || g.nc > QC_MAX_CONTROLS) return qc_fail(QC_ERR_ARG, "gate with nc=%d", g.nc);
  if (int rc = qc_check_qubits(n, g.qubits, k, g.controls, g.cstates, g.nc)) return rc;
  R.k = k;
  R.nc = g.nc;
  for (int i = 0; i < k; i++) R.t[i] = g.qubits[i];
  for (int i = 0; i < g.nc; i++) { R.c[i] = g.controls[i]; R.cs[i] = g.cstates[i]; }
  return QC_OK;
}

void to_op(int n, const Resolved& R, qc_op& op) {
  op.kind = QC_OP_MATRIX;
  op.k = R.k;
  op.nc = R.nc;
  for (int i = 0; i < R.k; i++) op.tpos[i] = n - 1 - R.t[i];
  for (int i = 0; i < R.nc; i++) { op.cpos[i] = n - 1 - R.c[i]; op.cval[i] = R.cs[i]; }
  const size_t D = (size_t)1 << R.k;
  for (size_t i = 0; i < D * D; i++) { op.U[2 * i] = R.U[i].real(); op.U[2 * i + 1] = R.U[i].imag(); }
}

// ---------------------------------------------------------------- fusion
// A fused block: qubits q[0..m) (q[0] = most significant bit of the block
// index) and its 2^m x 2^m unitary, accumulated in FP64.  A block's columns
// are states of an m-qubit register, so appending a gate applies that gate
// to every column.
struct Block {
  std::vector<int> q;
  std::vector<cd> M;     // row-major
  int ngates = 0;
  int first = -1;        // index of the first gate (single-gate blocks keep it)
};

int local_index(const Block& b, int qubit) {
  for (size_t i = 0; i < b.q.size(); i++) if (b.q[i] == qubit) return (int)i;
  return -1;
}

// Apply a resolved gate to the block's matrix (left-multiply): for every row
// group the gate connects (target bits of the row index running, control bits
// at their states) the group's rows are replaced by U times them, whole rows at
// a time.
void block_apply(Block& b, const Resolved& R) {
  const int m = (int)b.q.size();
  const int d = 1 << m;
  int tl[QC_MAX_TARGETS], cl[QC_MAX_CONTROLS];
  for (int i = 0; i < R.k; i++) tl[i] = m - 1 - local_index(b, R.t[i]);   // bit positions in block index
  for (int i = 0; i < R.nc; i++) cl[i] = m - 1 - local_index(b, R.c[i]);
  const int kd = 1 << R.k;
  std::vector<cd> rows((size_t)kd * d);
  for (int x = 0; x < d; x++) {
    bool base = true;
    for (int i = 0; i < R.k; i++) if ((x >> tl[i]) & 1) base = false;
    for (int i = 0; i < R.nc; i++) if (((x >> cl[i]) & 1) != R.cs[i]) base = false;
    if (!base) continue;
    int idx[1 << QC_MAX_TARGETS];
    for (int r = 0; r < kd; r++) {
      int y = x;
      for (int i = 0; i < R.k; i++) if ((r >> (R.k - 1 - i)) & 1) y |= 1 << tl[i];
      idx[r] = y;
      std::copy(b.M.begin() + (size_t)y * d, b.M.begin() + (size_t)(y + 1) * d, rows.begin() + (size_t)r * d);
    }
    for (int r = 0; r < kd; r++) {
      cd* out = &b.M[(size_t)idx[r] * d];
      std::fill(out, out + d, cd(0));
      for (int c = 0; c < kd; c++) {
        const cd u = R.U[(size_t)r * kd + c];
        if (u == cd(0)) continue;
        const cd* in = &rows[(size_t)c * d];
        for (int j = 0; j < d; j++) out[j] += u * in[j];
      }
    }
  }
  b.ngates++;
}


// A planned entry: a block's qubits (q[0] = most significant bit of its
// matrix) and its gates in application order.  One gate: applied as it is
// (its structured kernel); more: one dense block, built once the plan is
// chosen.  The planners below work on qubit sets and gate lists only.
struct Planned {
  std::vector<int> q;
  std::vector<int> gates;
  int first = -1;         // smallest gate index (flush order)
};

std::vector<int> gate_qubits(const Resolved& R) {
  std::vector<int> qs(R.t, R.t + R.k);
  qs.insert(qs.end(), R.c, R.c + R.nc);
  return qs;
}

bool has_qubit(const std::vector<int>& qs, int q) { return std::find(qs.begin(), qs.end(), q) != qs.end(); }

// Greedy fusion with several open blocks on disjoint qubit sets: a gate joins
// (and merges) the open blocks it touches when the union has at most kmax
// qubits; otherwise touched blocks are emitted, largest first, until it fits.
// Blocks on disjoint qubits commute, so emission order stays valid.
void fuse(int n, const std::vector<Resolved>& gates, int kmax, std::vector<Planned>& out) {
  std::vector<Planned> open;
  std::vector<int> owner(n, -1);   // qubit -> open block index
  auto emit = [&](int bi) {
    Planned& b = open[bi];
    for (int q : b.q) owner[q] = -1;
    out.push_back(std::move(b));
    b = Planned();
  };
  for (int gi = 0; gi < (int)gates.size(); gi++) {
    const std::vector<int> qs = gate_qubits(gates[gi]);
    std::vector<int> touched;
    int width = 0;
    for (int q : qs) {
      const int o = owner[q];
      if (o < 0) width++;
      else if (std::find(touched.begin(), touched.end(), o) == touched.end()) touched.push_back(o);
    }
    for (int o : touched) width += (int)open[o].q.size();
    if ((int)qs.size() > kmax) {          // wider than a block: applied on its own
      for (int o : touched) emit(o);
      Planned e;
      e.q = qs;
      e.gates = {gi};
      e.first = gi;
      out.push_back(std::move(e));
      continue;
    }
    if (width > kmax) {
      // Emit touched blocks, the one with the most qubits first, until the gate
      // and the remaining ones fit in one block.  Emitting a block early is
      // exact: its gates precede this gate and act on qubits no other open
      // block holds.  (Emitting every touched block instead: brickwork n=30,
      // k=5 took 229 blocks; this rule 142.)
      std::sort(touched.begin(), touched.end(),
                [&](int a, int b) { return open[a].q.size() > open[b].q.size() || (open[a].q.size() == open[b].q.size() && a < b); });
      while (width > kmax && !touched.empty()) {
        const int o = touched.front();
        width -= (int)open[o].q.size();
        for (int q : qs) if (has_qubit(open[o].q, q)) width++;   // its qubits in the gate become free
        emit(o);
        touched.erase(touched.begin());
      }
    }
    // merge the touched blocks (if any) into one; their gates commute (disjoint qubits)
    Planned nb;
    std::sort(touched.begin(), touched.end());
    for (int o : touched) {
      for (int q : open[o].q) { nb.q.push_back(q); owner[q] = -1; }
      nb.gates.insert(nb.gates.end(), open[o].gates.begin(), open[o].gates.end());
      if (nb.first < 0 || open[o].first < nb.first) nb.first = open[o].first;
      open[o] = Planned();
    }
    for (int q : qs) if (!has_qubit(nb.q, q)) nb.q.push_back(q);
    nb.gates.push_back(gi);
    if (nb.first < 0) nb.first = gi;
    int slot = -1;
    for (int i = 0; i < (int)open.size(); i++) if (open[i].q.empty()) { slot = i; break; }
    if (slot < 0) { slot = (int)open.size(); open.emplace_back(); }
    open[slot] = std::move(nb);
    for (int q : open[slot].q) owner[q] = slot;
  }
  // flush in order of first gate
  std::vector<int> rest;
  for (int i = 0; i < (int)open.size(); i++) if (!open[i].q.empty()) rest.push_back(i);
  std::sort(rest.begin(), rest.end(), [&](int a, int b) { return open[a].first < open[b].first; });
  for (int i : rest) emit(i);
}

// Fusion from the dependency front, one block at a time: a gate is ready when
// every earlier gate on its qubits has been taken.  A block starts at the
// earliest remaining gate (always ready), takes every ready gate inside its
// qubit set, and widens by the qubits of the earliest ready gate that keeps it
// within kmax, until neither is possible.  Gates taken in this order respect
// every qubit's gate order, so the emitted sequence equals the circuit.
void fuse_front(int n, const std::vector<Resolved>& gates, int kmax, std::vector<Planned>& out) {
  const int G = (int)gates.size();
  std::vector<std::vector<int>> on_q(n), qs_of(G);
  for (int i = 0; i < G; i++) {
    qs_of[i] = gate_qubits(gates[i]);
    for (int q : qs_of[i]) on_q[q].push_back(i);
  }
  std::vector<int> pos(n, 0);
  std::vector<char> taken(G, 0);
  auto ready = [&](int i) {
    if (taken[i]) return false;
    for (int q : qs_of[i]) if (on_q[q][pos[q]] != i) return false;
    return true;
  };
  auto take = [&](int i, Planned& b) {
    taken[i] = 1;
    for (int q : qs_of[i]) pos[q]++;
    b.gates.push_back(i);
  };
  int next = 0;
  while (true) {
    while (next < G && taken[next]) next++;
    if (next >= G) break;
    const int seed = next;                       // all its predecessors are taken
    Planned b;
    b.q = qs_of[seed];
    b.first = seed;
    if ((int)qs_of[seed].size() > kmax) {
      take(seed, b);
      out.push_back(std::move(b));
      continue;
    }
    for (bool grown = true; grown;) {
      // every ready gate inside the block's qubits
      for (bool more = true; more;) {
        more = false;
        for (size_t j = 0; j < b.q.size(); j++) {
          const int q = b.q[j];
          while (pos[q] < (int)on_q[q].size()) {
            const int i = on_q[q][pos[q]];
            bool inside = ready(i);
            for (int qq : qs_of[i]) if (inside && !has_qubit(b.q, qq)) inside = false;
            if (!inside) break;
            take(i, b);
            more = true;
          }
        }
      }
      // widen by the earliest ready gate on the block's qubits that fits
      grown = false;
      int best = -1;
      for (size_t j = 0; j < b.q.size(); j++) {
        const int q = b.q[j];
        if (pos[q] >= (int)on_q[q].size()) continue;
        const int i = on_q[q][pos[q]];
        if (!ready(i)) continue;
        int width = (int)b.q.size();
        for (int qq : qs_of[i]) if (!has_qubit(b.q, qq)) width++;
        if (width <= kmax && (best < 0 || i < best)) best = i;
      }
      if (best >= 0) {
        for (int qq : qs_of[best]) if (!has_qubit(b.q, qq)) b.q.push_back(qq);
        grown = true;
      }
    }
    out.push_back(std::move(b));
  }
}

// Merge pass over a plan: each entry moves back past earlier entries on
// disjoint qubits (they commute with it) and joins the nearest earlier entry
// whose union with it has at most kmax qubits; it stays where it is when it
// reaches an entry it shares a qubit with and their union is wider.  Repeated
// until nothing merges.  A merged entry becomes a dense block; unmerged single
// gates stay as they are, so structured kernels (permutations, phases) keep
// serving them.
void merge_pass(int kmax, std::vector<Planned>& em) {
  for (bool changed = true; changed;) {
    changed = false;
    std::vector<Planned> out;
    for (Planned& e : em) {
      int target = -1;
      for (int i = (int)out.size() - 1; i >= 0; i--) {
        int uni = (int)out[i].q.size(), shared = 0;
        for (int q : e.q) {
          if (has_qubit(out[i].q, q)) shared++;
          else uni++;
        }
        if ((int)e.q.size() <= kmax && uni <= kmax) { target = i; break; }
        if (shared) break;
      }
      if (target < 0) {
        out.push_back(std::move(e));
        continue;
      }
      // out[target]'s gates, then e's (e commutes with every entry in between)
      for (int q : e.q) if (!has_qubit(out[target].q, q)) out[target].q.push_back(q);
      out[target].gates.insert(out[target].gates.end(), e.gates.begin(), e.gates.end());
      changed = true;
    }
    em.swap(out);
  }
}

}  // namespace

int qc_gate_to_op(int n, const qc_gate& g, qc_op& op) {
  Resolved R;
  if (int rc = resolve(n, g, R)) return rc;
  to_op(n, R, op);
  return QC_OK;
}

namespace {
int plan_ops(int n, const qc_gate* gates, int ngates, int fuse_k, std::vector<qc_op>& ops, bool phase_runs);
}

int qc_plan_ops(int n, const qc_gate* gates, int ngates, int fuse_k, std::vector<qc_op>& ops, bool phase_runs) {
  return plan_ops(n, gates, ngates, fuse_k, ops, phase_runs);
}

namespace {
// A (controlled) phase gate whose phase applies when all of its qubits are 1:
// diag(1, e^{i theta}) on the target, controls in state 1.  Returns the qubit
// set (1 or 2 qubits) and theta, or false.
bool phase_gate(const Resolved& R, int* qs, int* nq, double* theta) {
  if (R.k != 1 || R.nc > 1) return false;
  for (int i = 0; i < R.nc; i++) if (R.cs[i] != 1) return false;
  const cd u00 = R.U[0], u01 = R.U[1], u10 = R.U[2], u11 = R.U[3];
  if (u01 != cd(0) || u10 != cd(0) || u00 != cd(1)) return false;
  if (std::abs(std::abs(u11) - 1.0) > 1e-14) return false;
  *theta = std::arg(u11);
  *nq = 0;
  qs[(*nq)++] = R.t[0];
  for (int i = 0; i < R.nc; i++) qs[(*nq)++] = R.c[i];
  return true;
}

// An uncontrolled SWAP: the 4x4 permutation exchanging |01> and |10>.
bool swap_gate(const Resolved& R) {
  if (R.k != 2 || R.nc != 0) return false;
  static const int perm[4] = {0, 2, 1, 3};
  for (int r = 0; r < 4; r++)
    for (int c = 0; c < 4; c++)
      if (R.U[r * 4 + c] != cd(c == perm[r] ? 1.0 : 0.0)) return false;
  return true;
}

void emit_matrix_segment(int n, const std::vector<Resolved>& res, int begin, int end, int fuse_k,
                         std::vector<qc_op>& ops) {
  if (begin >= end) return;
  std::vector<Resolved> seg(res.begin() + begin, res.begin() + end);
  // two planners, each followed by the merge pass; the plan with fewer sweeps
  // is kept (ties: the first); only its blocks' matrices are built
  const int kmax = std::min(fuse_k, n);
  std::vector<Planned> em, em2;
  fuse(n, seg, kmax, em);
  merge_pass(kmax, em);
  fuse_front(n, seg, kmax, em2);
  merge_pass(kmax, em2);
  if (em2.size() < em.size()) em.swap(em2);
  for (const Planned& p : em) {
    qc_op op;
    if (p.gates.size() == 1) { to_op(n, seg[p.gates[0]], op); ops.push_back(op); continue; }
    Block b;
    b.q = p.q;
    const size_t d = (size_t)1 << p.q.size();
    b.M.assign(d * d, cd(0));
    for (size_t i = 0; i < d; i++) b.M[i * d + i] = 1;
    for (int g : p.gates) block_apply(b, seg[g]);
    Resolved R;
    R.k = (int)b.q.size();
    R.nc = 0;
    for (int j = 0; j < R.k; j++) R.t[j] = b.q[j];
    R.U = b.M;
    to_op(n, R, op);
    ops.push_back(op);
  }
}

// Build the launch plan (shared by qc_apply_circuit, qc_fuse_plan and the batch path).
int plan_ops(int n, const qc_gate* gates, int ngates, int fuse_k, std::vector<qc_op>& ops, bool phase_runs) {
  if (ngates < 0 || (ngates > 0 && !gates)) return qc_fail(QC_ERR_ARG, "invalid gate list");
  if (fuse_k < 0 || fuse_k > QC_MAX_TARGETS) return qc_fail(QC_ERR_ARG, "fuse_k=%d out of range 0..5", fuse_k);
  std::vector<Resolved> res(ngates);
  for (int i = 0; i < ngates; i++)
    if (int rc = resolve(n, gates[i], res[i])) return qc_fail(rc, "gate %d: %s", i, qc_last_error());
  ops.clear();
  if (fuse_k >= 2) {
    int seg_begin = 0;
    int i = 0;
    while (i < ngates) {
      // longest run of phase gates from i that share a qubit (the anchor)
      int qs[2], nq;
      double th;
      int j = i;
      uint64_t common = 0;
      if (phase_runs && phase_gate(res[i], qs, &nq, &th)) {
        common = 0;
        for (int t = 0; t < nq; t++) common |= 1ull << qs[t];
        j = i + 1;
        std::vector<int> lin;
        while (j < ngates && phase_gate(res[j], qs, &nq, &th)) {
          uint64_t s = 0;
          for (int t = 0; t < nq; t++) s |= 1ull << qs[t];
          if (!(common & s)) break;
          const uint64_t c2 = common & s;
          // distinct linear qubits (all but the anchor) must stay within QC_MAX_LIN
          int distinct = 0;
          uint64_t seen = 0;
          for (int g = i; g <= j; g++) {
            int q2[2], n2;
            double t2;
            phase_gate(res[g], q2, &n2, &t2);
            for (int t = 0; t < n2; t++) seen |= 1ull << q2[t];
          }
          distinct = __builtin_popcountll(seen) - 1;
          if (distinct > QC_MAX_LIN) break;
          common = c2;
          j++;
        }
      }
      // longest run of SWAPs on disjoint qubit pairs from i: one bit permutation
      int js = i;
      uint64_t used = 0;
      while (phase_runs && js < ngates && swap_gate(res[js])) {
        const uint64_t pr = (1ull << res[js].t[0]) | (1ull << res[js].t[1]);
        if (used & pr) break;
        used |= pr;
        js++;
      }
      if (js - i >= 2) {
        emit_matrix_segment(n, res, seg_begin, i, fuse_k, ops);
        qc_op op;
        std::memset(&op, 0, sizeof(op));
        op.kind = QC_OP_PERMUTE;
        for (int g = i; g < js; g++) {
          op.perm_a[op.nperm] = n - 1 - res[g].t[0];
          op.perm_b[op.nperm] = n - 1 - res[g].t[1];
          op.nperm++;
        }
        ops.push_back(op);
        i = js;
        seg_begin = js;
        continue;
      }
      if (j - i >= 2) {
        emit_matrix_segment(n, res, seg_begin, i, fuse_k, ops);
        const int anchor = __builtin_ctzll(common);   // a qubit shared by every gate of the run
        qc_op op;
        std::memset(&op, 0, sizeof(op));
        op.kind = QC_OP_LINEAR_PHASE;
        op.anchor = n - 1 - anchor;
        double lin[64] = {0};
        uint64_t linmask = 0;
        for (int g = i; g < j; g++) {
          phase_gate(res[g], qs, &nq, &th);
          int other = -1;
          for (int t = 0; t < nq; t++) if (qs[t] != anchor) other = qs[t];
          if (other < 0) op.theta0 += th;
          else { lin[other] += th; linmask |= 1ull << other; }
        }
        for (int q = 0; q < n; q++)
          if ((linmask >> q) & 1) { op.lin_pos[op.nlin] = n - 1 - q; op.lin_theta[op.nlin] = lin[q]; op.nlin++; }
        // A lone 1-qubit op on the anchor just before the run (the H of a QFT
        // stage, Fig. 1) joins the run's sweep: U on the anchor pair, then the
        // phase.  The merged kernel needs the anchor at bit 4 or above.
        if (!ops.empty() && op.anchor >= 4) {
          const qc_op& last = ops.back();
          if (last.kind == QC_OP_MATRIX && last.k == 1 && last.nc == 0 && last.tpos[0] == op.anchor) {
            op.pre = 1;
            op.k = 1;
            op.tpos[0] = op.anchor;
            std::memcpy(op.U, last.U, sizeof(double) * 8);
            ops.pop_back();
          }
        }
        ops.push_back(op);
        i = j;
        seg_begin = j;
      } else {
        i++;
      }
    }
    emit_matrix_segment(n, res, seg_begin, ngates, fuse_k, ops);
  } else {
    ops.resize(ngates);
    for (int i = 0; i < ngates; i++) to_op(n, res[i], ops[i]);
  }
  return QC_OK;
}
}  // namespace

extern "C" int qc_fuse_plan(int n, const qc_gate* gates, int ngates, int fuse_k, qc_block* blocks,
                            int max_blocks, int* nblocks) {
  if (n < 1 || n > 36) return qc_fail(QC_ERR_ARG, "n=%d out of range 1..36", n);
  if (!nblocks) return qc_fail(QC_ERR_ARG, "nblocks is NULL");
  std::vector<qc_op> ops;
  if (int rc = plan_ops(n, gates, ngates, fuse_k, ops, true)) return rc;
  *nblocks = (int)ops.size();
  if ((int)ops.size() > max_blocks || (!blocks && !ops.empty()))
    return qc_fail(QC_ERR_ARG, "plan needs %d blocks, buffer holds %d", (int)ops.size(), max_blocks);
  for (size_t i = 0; i < ops.size(); i++) {
    const qc_op& op = ops[i];
    qc_block& b = blocks[i];
    std::memset(&b, 0, sizeof(b));
    if (op.kind == QC_OP_PERMUTE) {   // pairs of qubits in lin_qubits
      b.kind = 2;
      b.nlin = 2 * op.nperm;
      for (int j = 0; j < op.nperm; j++) {
        b.lin_qubits[2 * j] = n - 1 - op.perm_a[j];
        b.lin_qubits[2 * j + 1] = n - 1 - op.perm_b[j];
      }
      continue;
    }
    if (op.kind == QC_OP_LINEAR_PHASE) {
      b.kind = 1;
      b.anchor = n - 1 - op.anchor;
      b.nlin = op.nlin;
      for (int j = 0; j < op.nlin; j++) { b.lin_qubits[j] = n - 1 - op.lin_pos[j]; b.lin_theta[j] = op.lin_theta[j]; }
      b.theta0 = op.theta0;
      if (op.pre) {                  // the 2x2 matrix on the anchor applied first
        b.k = 1;
        b.qubits[0] = b.anchor;
        std::memcpy(b.U, op.U, sizeof(double) * 8);
      }
      continue;
    }
    b.k = op.k;
    for (int j = 0; j < op.k; j++) b.qubits[j] = n - 1 - op.tpos[j];
    b.nc = op.nc;
    for (int j = 0; j < op.nc; j++) { b.controls[j] = n - 1 - op.cpos[j]; b.cstates[j] = op.cval[j]; }
    const size_t D = (size_t)1 << op.k;
    std::memcpy(b.U, op.U, sizeof(double) * 2 * D * D);
  }
  return QC_OK;
}

extern "C" int qc_apply_circuit(qc_state* s, const qc_gate* gates, int ngates, const qc_opts* opts) {
  if (int rc = qc_check_state(s)) return rc;
  qc_opts o;
  std::memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  if (o.use_graph && s->stream == nullptr) return qc_fail(QC_ERR_ARG, "graph capture needs a non-default stream (qc_set_stream)");

  std::vector<qc_op> ops;
  if (int rc = plan_ops(s->n, gates, ngates, o.fuse_k, ops, true)) return rc;
  if (o.nlaunch) *o.nlaunch = (int)ops.size();

  std::vector<cudaEvent_t> ev;
  if (o.gate_ms) {
    ev.resize(ops.size() + 1);
    for (auto& e : ev) QC_CUDA(cudaEventCreate(&e));
  }
  cudaGraph_t graph = nullptr;
  if (o.use_graph) QC_CUDA(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
  int rc = QC_OK;
  if (o.gate_ms && !o.use_graph) cudaEventRecord(ev[0], s->stream);
  for (size_t i = 0; i < ops.size() && rc == QC_OK; i++) {
    rc = qc_launch_op(s, ops[i]);
    if (o.gate_ms && !o.use_graph) cudaEventRecord(ev[i + 1], s->stream);
  }
  if (o.use_graph) {
    cudaError_t e = cudaStreamEndCapture(s->stream, &graph);
    if (rc == QC_OK && e != cudaSuccess) rc = qc_cuda_fail(e, "cudaStreamEndCapture");
    if (rc == QC_OK) {
      cudaGraphExec_t exec = nullptr;
      e = cudaGraphInstantiate(&exec, graph, 0);
      if (e != cudaSuccess) rc = qc_cuda_fail(e, "cudaGraphInstantiate");
      else {
        if (o.gate_ms) cudaEventRecord(ev[0], s->stream);
        e = cudaGraphLaunch(exec, s->stream);
        if (e != cudaSuccess) rc = qc_cuda_fail(e, "cudaGraphLaunch");
        if (o.gate_ms) cudaEventRecord(ev[ops.size()], s->stream);
        cudaGraphExecDestroy(exec);
      }
    }
    if (graph) cudaGraphDestroy(graph);
  }
  if (o.gate_ms && rc == QC_OK) {
    cudaError_t e = cudaEventSynchronize(ev.back());
    if (e != cudaSuccess) rc = qc_cuda_fail(e, "cudaEventSynchronize");
    for (size_t i = 0; i < ops.size() && rc == QC_OK; i++) {
      float ms = 0.f;
      if (o.use_graph) {   // only the whole replay is timed; spread evenly
        if (i == 0) cudaEventElapsedTime(&ms, ev[0], ev[ops.size()]);
        o.gate_ms[i] = 0.f;
        if (i == 0) for (size_t j = 0; j < ops.size(); j++) o.gate_ms[j] = ms / ops.size();
      } else {
        cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
        o.gate_ms[i] = ms;
      }
    }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  if (o.gate_ms && rc == QC_OK) rc = qc_take_device_status("qc_apply_circuit");
  return rc;
}
