// qc_shard.cu -- one state split over 2^g shards (ranks): exchange planner
// and the shard kernels that move amplitudes between shards.
//
// Layout.  The g most significant qubits (qubits 0 .. g-1, Definition 1) are
// global: rank r holds the 2^(n-g) amplitudes whose top g index bits equal r,
// as an (n-g)-qubit state whose qubit j is qubit g + j of the whole register.
// Global qubit p is bit g-1-p of the rank.
//
// A gate whose targets are all local runs on every shard unchanged (qubits
// renumbered); a control on a global qubit becomes a condition on the rank.
// A target on a global qubit needs its amplitude pairs on one rank: the
// planner first exchanges that global qubit with a local one -- swapping
// index bits G (global) and L (local) of every amplitude moves exactly the
// amplitudes whose two bits differ, i.e. rank r sends the half of its shard
// with bit L = 1 - bit_G(r) to the rank r ^ (1 << bit) and receives the
// partner's half into the same slots -- and tracks the resulting
// logical-to-physical qubit permutation.  The local qubit is the one whose
// next use lies furthest ahead (Belady's rule).  An uncontrolled SWAP gate
// moves no data at all: it only exchanges two entries of the permutation.
// At the end the identity layout is restored by exchanges (global positions)
// and local SWAP gates.
#include <algorithm>
#include <cstring>
#include <vector>

#include "qc_common.cuh"

namespace {

struct Planner {
  int n, g;
  std::vector<int> perm, inv;              // logical -> physical, physical -> logical
  std::vector<qc_shard_step>* out;
  int count = 0;

  void emit(const qc_shard_step& s) {
    if (out) out->push_back(s);
    count++;
  }
  // exchange physical global position p with physical local position x
  void exchange(int p, int x) {
    qc_shard_step s;
    std::memset(&s, 0, sizeof(s));
    s.kind = QC_SHARD_EXCHANGE;
    s.rank_bit = g - 1 - p;
    s.local_qubit = x - g;
    emit(s);
    const int lp = inv[p], lx = inv[x];
    perm[lp] = x;
    perm[lx] = p;
    inv[p] = lx;
    inv[x] = lp;
  }
  void local_swap_gate(int x, int y) {      // SWAP of two physical local positions, on every rank
    qc_shard_step s;
    std::memset(&s, 0, sizeof(s));
    s.kind = QC_SHARD_GATE;
    s.gate.kind = QC_GATE_SWAP;
    s.gate.nq = 2;
    s.gate.qubits[0] = x - g;
    s.gate.qubits[1] = y - g;
    emit(s);
    const int lx = inv[x], ly = inv[y];
    perm[lx] = y;
    perm[ly] = x;
    inv[x] = ly;
    inv[y] = lx;
  }
};

int gate_width(const qc_gate& gt) {
  if (gt.kind == QC_GATE_MATRIX) return gt.nq;
  return gt.kind == QC_GATE_SWAP ? 2 : 1;
}

int plan(int n, int g, const qc_gate* gates, int ngates, std::vector<qc_shard_step>* out, int* count) {
  if (n < 2 || n > 36) return qc_fail(QC_ERR_ARG, "n=%d out of range 2..36", n);
  if (g < 1 || g > 16 || g >= n) return qc_fail(QC_ERR_ARG, "g=%d global qubits: need 1 <= g <= 16, g < n", g);
  if (ngates < 0 || (ngates > 0 && !gates)) return qc_fail(QC_ERR_ARG, "invalid gate list");
  // validate and collect the next uses of every logical qubit
  std::vector<std::vector<int>> uses(n);
  for (int i = 0; i < ngates; i++) {
    const qc_gate& gt = gates[i];
    const int k = gate_width(gt);
    if (gt.kind < QC_GATE_MATRIX || gt.kind > QC_GATE_SWAP) return qc_fail(QC_ERR_ARG, "gate %d: unknown kind %d", i, gt.kind);
    if (gt.nq != k || k < 1 || k > QC_MAX_TARGETS) return qc_fail(QC_ERR_ARG, "gate %d: nq=%d", i, gt.nq);
    if (gt.kind == QC_GATE_MATRIX && !gt.matrix) return qc_fail(QC_ERR_ARG, "gate %d: matrix is NULL", i);
    if (int rc = qc_check_qubits(n, gt.qubits, k, gt.controls, gt.cstates, gt.nc)) return rc;
    if (k > n - g) return qc_fail(QC_ERR_ARG, "gate %d: %d targets do not fit %d local qubits", i, k, n - g);
    for (int t = 0; t < k; t++) uses[gt.qubits[t]].push_back(i);
    for (int c = 0; c < gt.nc; c++) uses[gt.controls[c]].push_back(i);
  }
  std::vector<size_t> cursor(n, 0);
  auto next_use = [&](int logical, int after) {
    auto& u = uses[logical];
    size_t& c = cursor[logical];
    while (c < u.size() && u[c] <= after) c++;
    return c < u.size() ? u[c] : ngates + 1;
  };
  Planner P;
  P.n = n;
  P.g = g;
  P.out = out;
  P.perm.resize(n);
  P.inv.resize(n);
  for (int q = 0; q < n; q++) P.perm[q] = P.inv[q] = q;
  for (int i = 0; i < ngates; i++) {
    const qc_gate& gt = gates[i];
    const int k = gate_width(gt);
    if (gt.kind == QC_GATE_SWAP && gt.nc == 0) {    // relabel only
      const int a = gt.qubits[0], b = gt.qubits[1];
      std::swap(P.perm[a], P.perm[b]);
      P.inv[P.perm[a]] = a;
      P.inv[P.perm[b]] = b;
      continue;
    }
    // bring every target to a local position
    for (int t = 0; t < k; t++) {
      const int p = P.perm[gt.qubits[t]];
      if (p >= g) continue;
      int best = -1, best_next = -1;
      for (int x = g; x < n; x++) {
        const int lx = P.inv[x];
        bool busy = false;
        for (int u = 0; u < k && !busy; u++) busy = gt.qubits[u] == lx;
        for (int u = 0; u < gt.nc && !busy; u++) busy = gt.controls[u] == lx;
        if (busy) continue;
        const int nu = next_use(lx, i);
        if (nu > best_next) { best_next = nu; best = x; }
      }
      if (best < 0) return qc_fail(QC_ERR_ARG, "gate %d does not fit the %d local qubits", i, n - g);
      P.exchange(p, best);
    }
    qc_shard_step s;
    std::memset(&s, 0, sizeof(s));
    s.kind = QC_SHARD_GATE;
    s.gate = gt;
    s.gate.nc = 0;
    for (int t = 0; t < k; t++) s.gate.qubits[t] = P.perm[gt.qubits[t]] - g;
    for (int c = 0; c < gt.nc; c++) {
      const int p = P.perm[gt.controls[c]];
      if (p < g) {
        s.rank_mask |= 1u << (g - 1 - p);
        if (gt.cstates[c]) s.rank_val |= 1u << (g - 1 - p);
      } else {
        s.gate.controls[s.gate.nc] = p - g;
        s.gate.cstates[s.gate.nc] = gt.cstates[c];
        s.gate.nc++;
      }
    }
    P.emit(s);
  }
  // restore the identity layout: global positions by exchanges, then local ones by SWAP gates
  for (int l = 0; l < g; l++) {
    const int p = P.perm[l];
    if (p == l) continue;
    if (p >= g) {
      P.exchange(l, p);
    } else {
      const int x = g;                              // any local position serves as the stop-over
      P.exchange(p, x);
      P.exchange(l, x);
    }
  }
  for (int l = g; l < n; l++)
    if (P.perm[l] != l) P.local_swap_gate(P.perm[l], l);
  *count = P.count;
  return QC_OK;
}

// ---------------------------------------------------------------- kernels
// Half of a shard: the amplitudes whose bit at position pb (pb = n_local - 1 -
// local_qubit) equals `bit`; entry j of the half is index insert_zero(j, pb) |
// bit << pb, counted in units of U: 32-byte vectors (two complex128 or four
// complex64 amplitudes that share every bit but the lowest one or two) when pb
// leaves them whole, else 16- or 8-byte units.  Two units per thread and
// iteration, both loads issued first.
struct alignas(32) U32 { uint4 a, b; };

template <class U>
__device__ __forceinline__ U ld_unit(const U* p) { return *p; }
template <>
__device__ __forceinline__ U32 ld_unit<U32>(const U32* p) {
  const vec32 v = qc_ld32(p);
  U32 u;
  u.a = make_uint4(v.w[0], v.w[1], v.w[2], v.w[3]);
  u.b = make_uint4(v.w[4], v.w[5], v.w[6], v.w[7]);
  return u;
}
template <class U>
__device__ __forceinline__ void st_unit(U* p, const U& u) { *p = u; }
template <>
__device__ __forceinline__ void st_unit<U32>(U32* p, const U32& u) {
  vec32 v;
  v.w[0] = u.a.x; v.w[1] = u.a.y; v.w[2] = u.a.z; v.w[3] = u.a.w;
  v.w[4] = u.b.x; v.w[5] = u.b.y; v.w[6] = u.b.z; v.w[7] = u.b.w;
  qc_st32(p, v);
}

template <class U>
__global__ void __launch_bounds__(256)
k_shard_swap(U* __restrict__ a, U* __restrict__ b, uint64_t nhalf, int pb, uint64_t abit, uint64_t bbit) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nhalf; j += 2 * stride) {
    const bool two = j + stride < nhalf;
    const uint64_t b0 = qc_insert_zero(j, pb), b1 = two ? qc_insert_zero(j + stride, pb) : b0;
    const uint64_t ia0 = b0 | (abit << pb), ib0 = b0 | (bbit << pb);
    const uint64_t ia1 = b1 | (abit << pb), ib1 = b1 | (bbit << pb);
    const U x0 = ld_unit(a + ia0), y0 = ld_unit(b + ib0);
    const U x1 = ld_unit(a + ia1), y1 = ld_unit(b + ib1);
    st_unit(a + ia0, y0);
    st_unit(b + ib0, x0);
    if (two) {
      st_unit(a + ia1, y1);
      st_unit(b + ib1, x1);
    }
  }
}

template <class U>
__global__ void __launch_bounds__(256)
k_shard_pack(const U* __restrict__ s, U* __restrict__ buf, uint64_t nhalf, int pb, uint64_t bit) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nhalf; j += stride)
    st_unit(buf + j, ld_unit(s + (qc_insert_zero(j, pb) | (bit << pb))));
}

template <class U>
__global__ void __launch_bounds__(256)
k_shard_unpack(U* __restrict__ s, const U* __restrict__ buf, uint64_t nhalf, int pb, uint64_t bit) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nhalf; j += stride)
    st_unit(s + (qc_insert_zero(j, pb) | (bit << pb)), ld_unit(buf + j));
}

struct HalfGeom {
  int ubytes;         // 32, 16 or 8 bytes per unit
  uint64_t nhalf;     // units per half
  int pb;             // bit position in units
};

int half_geom(const qc_state* s, int local_qubit, HalfGeom& h) {
  if (local_qubit < 0 || local_qubit >= s->n) return qc_fail(QC_ERR_ARG, "local qubit %d out of range 0..%d", local_qubit, s->n - 1);
  const int pb = s->n - 1 - local_qubit;              // amplitude units
  const int lv = s->dtype == QC_C128 ? 1 : 2;         // log2 amplitudes per 32-byte unit
  const int l16 = s->dtype == QC_C128 ? 0 : 1;        // log2 amplitudes per 16-byte unit
  if (pb >= lv && s->n - 1 >= lv) { h.ubytes = 32; h.pb = pb - lv; h.nhalf = 1ull << (s->n - 1 - lv); return QC_OK; }
  if (pb >= l16 && s->n - 1 >= l16) { h.ubytes = 16; h.pb = pb - l16; h.nhalf = 1ull << (s->n - 1 - l16); return QC_OK; }
  h.ubytes = 8;
  h.pb = pb;
  h.nhalf = 1ull << (s->n - 1);
  return QC_OK;
}

int grid_of(uint64_t work) {
  const uint64_t want = (work + 255) / 256;
  return (int)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)qc_num_sms() * 16));
}

}  // namespace

extern "C" int qc_shard_plan(int n, int g, const qc_gate* gates, int ngates, qc_shard_step* steps, int max_steps,
                             int* nsteps) {
  if (!nsteps) return qc_fail(QC_ERR_ARG, "nsteps is NULL");
  *nsteps = 0;
  std::vector<qc_shard_step> out;
  int count = 0;
  if (int rc = plan(n, g, gates, ngates, &out, &count)) return rc;
  *nsteps = count;
  if (!steps) return QC_OK;
  if (count > max_steps) return qc_fail(QC_ERR_ARG, "the plan has %d steps, more than max_steps=%d", count, max_steps);
  std::memcpy(steps, out.data(), sizeof(qc_shard_step) * (size_t)count);
  return QC_OK;
}

extern "C" int qc_shard_exchange(qc_state* a, qc_state* b, int local_qubit, int bit_a) {
  if (int rc = qc_check_state(a)) return rc;
  if (!b || !b->ptr) return qc_fail(QC_ERR_ARG, "state handle is NULL");
  if (a == b || a->ptr == b->ptr) return qc_fail(QC_ERR_ARG, "the two shards must be distinct");
  if (a->n != b->n || a->dtype != b->dtype) return qc_fail(QC_ERR_ARG, "shards differ in qubit count or dtype");
  if (bit_a != 0 && bit_a != 1) return qc_fail(QC_ERR_ARG, "bit_a must be 0 or 1");
  HalfGeom h;
  if (int rc = half_geom(a, local_qubit, h)) return rc;
  // a's half {bit = 1 - bit_a} trades places with b's half {bit = bit_a}
  const uint64_t abit = (uint64_t)(1 - bit_a), bbit = (uint64_t)bit_a;
  const int grid = grid_of(h.nhalf / 2 + 1);
  if (h.ubytes == 32)
    k_shard_swap<U32><<<grid, 256, 0, a->stream>>>((U32*)a->ptr, (U32*)b->ptr, h.nhalf, h.pb, abit, bbit);
  else if (h.ubytes == 16)
    k_shard_swap<uint4><<<grid, 256, 0, a->stream>>>((uint4*)a->ptr, (uint4*)b->ptr, h.nhalf, h.pb, abit, bbit);
  else
    k_shard_swap<uint2><<<grid, 256, 0, a->stream>>>((uint2*)a->ptr, (uint2*)b->ptr, h.nhalf, h.pb, abit, bbit);
  QC_LAUNCHED("k_shard_swap");
  return QC_OK;
}

extern "C" int qc_shard_pack(const qc_state* s, int local_qubit, int bit, void* dev_buf) {
  if (int rc = qc_check_state(s)) return rc;
  if (!dev_buf) return qc_fail(QC_ERR_ARG, "dev_buf is NULL");
  if (((uintptr_t)dev_buf) % 16 != 0) return qc_fail(QC_ERR_ARG, "dev_buf must be 16-byte aligned");
  if (bit != 0 && bit != 1) return qc_fail(QC_ERR_ARG, "bit must be 0 or 1");
  HalfGeom h;
  if (int rc = half_geom(s, local_qubit, h)) return rc;
  if (h.ubytes == 32 && ((uintptr_t)dev_buf) % 32 == 0)
    k_shard_pack<U32><<<grid_of(h.nhalf), 256, 0, s->stream>>>((const U32*)s->ptr, (U32*)dev_buf, h.nhalf, h.pb, (uint64_t)bit);
  else if (h.ubytes >= 16)
    k_shard_pack<uint4><<<grid_of(h.nhalf * (h.ubytes / 16)), 256, 0, s->stream>>>(
        (const uint4*)s->ptr, (uint4*)dev_buf, h.nhalf * (h.ubytes / 16), h.pb + (h.ubytes == 32), (uint64_t)bit);
  else
    k_shard_pack<uint2><<<grid_of(h.nhalf), 256, 0, s->stream>>>((const uint2*)s->ptr, (uint2*)dev_buf, h.nhalf, h.pb, (uint64_t)bit);
  QC_LAUNCHED("k_shard_pack");
  return QC_OK;
}

extern "C" int qc_shard_unpack(qc_state* s, int local_qubit, int bit, const void* dev_buf) {
  if (int rc = qc_check_state(s)) return rc;
  if (!dev_buf) return qc_fail(QC_ERR_ARG, "dev_buf is NULL");
  if (((uintptr_t)dev_buf) % 16 != 0) return qc_fail(QC_ERR_ARG, "dev_buf must be 16-byte aligned");
  if (bit != 0 && bit != 1) return qc_fail(QC_ERR_ARG, "bit must be 0 or 1");
  HalfGeom h;
  if (int rc = half_geom(s, local_qubit, h)) return rc;
  if (h.ubytes == 32 && ((uintptr_t)dev_buf) % 32 == 0)
    k_shard_unpack<U32><<<grid_of(h.nhalf), 256, 0, s->stream>>>((U32*)s->ptr, (const U32*)dev_buf, h.nhalf, h.pb, (uint64_t)bit);
  else if (h.ubytes >= 16)
    k_shard_unpack<uint4><<<grid_of(h.nhalf * (h.ubytes / 16)), 256, 0, s->stream>>>(
        (uint4*)s->ptr, (const uint4*)dev_buf, h.nhalf * (h.ubytes / 16), h.pb + (h.ubytes == 32), (uint64_t)bit);
  else
    k_shard_unpack<uint2><<<grid_of(h.nhalf), 256, 0, s->stream>>>((uint2*)s->ptr, (const uint2*)dev_buf, h.nhalf, h.pb, (uint64_t)bit);
  QC_LAUNCHED("k_shard_unpack");
  return QC_OK;
}
