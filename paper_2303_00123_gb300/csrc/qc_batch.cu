// qc_batch.cu -- many independent circuits in one persistent launch.
//
// Host: every circuit is planned (resolved, optionally fused into blocks of
// k <= 4 qubits) into ops {targets, controls, dense matrix}; all ops, matrices
// and per-circuit records go to one device allocation.  Two queues: circuits
// swept by teams, largest work (2^n * ops per member) first, and single-CTA
// circuits, smallest work first.
//
// Device: a persistent kernel with as many CTAs as fit at once (all of them
// co-resident).  A share of the CTAs proportional to the single-CTA work
// starts on that queue, the rest on the team queue; a CTA whose queue is empty
// takes from the other.  A CTA takes the next entry:
//   * shared-memory mode (state <= kSmemState bytes): one CTA builds the state
//     as |0...0> in shared memory, applies every op there (threads over the
//     op's groups, __syncthreads between ops) and writes the final state to
//     HBM once -- one pass over HBM for the whole circuit;
//   * global mode: a team of T CTAs (T = 1..16 by state size; the circuit has
//     T consecutive queue entries) initialises the state in place and sweeps it
//     op by op, each member taking 1/T of every op's groups, with a team
//     barrier (a per-circuit arrival counter) between ops.
// Deadlock freedom: the grid never exceeds the co-resident capacity, team
// entries are consecutive in their own queue and T <= 16 < grid, so at most
// one team is partly dequeued at any time and its missing members are the next
// team entries, taken by CTAs that finish work that waits on nothing
// unfinished (single-CTA circuits never wait).  Every barrier wait
// is bounded; a wait that gives up sets a status word (the host returns
// QC_ERR_TIMEOUT) and the team abandons that circuit.
// %globaltimer stamps give each circuit's completion time.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "qc_common.cuh"

namespace {

constexpr int kBT = 256;                 // threads per CTA
constexpr int kMaxK = 4;                 // widest op (fused block)
constexpr int kMaxD = 1 << kMaxK;
constexpr size_t kSmemState = 64 * 1024; // bytes of shared memory for a state

struct BOp {
  uint32_t coef;      // first matrix entry in the coef table
  uint8_t k;          // targets
  uint8_t nins;       // inserted positions (targets + controls)
  uint8_t tpos[kMaxK];
  uint8_t ins[QC_MAX_INS];
  uint64_t orval;     // control values
};

struct BCirc {
  uint64_t state;     // device address of the state
  uint32_t op0, nops; // op range
  int n;
  int smem;           // 1: shared-memory mode
  int team;           // CTAs working on this circuit (1 in shared-memory mode)
};

struct BEntry {
  uint32_t circ;      // circuit index
  uint32_t member;    // 0..team-1
};

struct BCtl {
  unsigned int queue;       // next entry of the team queue
  unsigned int queue2;      // next entry of the single-CTA queue
  int status;               // 0, or 1 when a team barrier gave up
  int skip_circ;            // test hook: this circuit's member `skip_member` never arrives (-1: off)
  int skip_member;
  unsigned long long spin_limit;
};

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Apply one op to a state held at `st` (shared or global memory), all
// threads; each thread loads UNR groups before computing them, so a CTA that
// sweeps a large state in global memory keeps enough loads in flight.
// State reads: shared memory, or global memory through L2 only (ld.global.cg):
// team members on other SMs write the state between ops, and L1 is not
// coherent across SMs, so a cached line could be stale after a team barrier.
template <bool GLOBAL, class T>
__device__ __forceinline__ T ld_state(const T* p) {
  if constexpr (GLOBAL) return __ldcg(p);
  else return *p;
}

template <class Ar, int K, bool GLOBAL>
__device__ __forceinline__ void apply_op(typename Ar::raw_t* st, const BOp& op, const typename Ar::coef_t* M,
                                         const uint64_t* moff, uint64_t g0, uint64_t g1) {
  constexpr int D = 1 << K;
  constexpr int UNR = D >= 8 ? 1 : 8 / D;
  for (uint64_t j0 = g0 + (uint64_t)threadIdx.x * UNR; j0 < g1; j0 += (uint64_t)kBT * UNR) {
    uint64_t b[UNR];
    typename Ar::val_t in[UNR][D];
#pragma unroll
    for (int u = 0; u < UNR; u++) {
      const uint64_t j = j0 + u < g1 ? j0 + u : j0;   // duplicates of j0 are read, never written
      uint64_t x = j;
      for (int i = 0; i < op.nins; i++) x = qc_insert_zero(x, op.ins[i]);
      b[u] = x | op.orval;
#pragma unroll
      for (int r = 0; r < D; r++) in[u][r] = Ar::from_raw(ld_state<GLOBAL>(st + b[u] + moff[r]));
    }
#pragma unroll
    for (int u = 0; u < UNR; u++) {
      if (u > 0 && j0 + u >= g1) break;
#pragma unroll
      for (int r = 0; r < D; r++) st[b[u] + moff[r]] = Ar::to_raw(Ar::template dot<D>(&M[r * D], in[u]));
    }
  }
}

// Team barrier: every member arrives once per phase; returns false when the
// bounded wait gave up (the status word is then set).
__device__ bool team_barrier(unsigned int* bar, unsigned int target, bool arrive, BCtl* ctl) {
  __syncthreads();
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    __threadfence();
    if (arrive) atomicAdd(bar, 1u);
    int ok = 1;
    unsigned long long it = 0;
    while (atomicAdd(bar, 0u) < target) {
      if (++it > ctl->spin_limit || atomicAdd(&ctl->status, 0) != 0) { ok = 0; break; }
      __nanosleep(128);
    }
    if (!ok) atomicExch(&ctl->status, 1);
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <class Ar>
__global__ void __launch_bounds__(kBT, 2)
k_batch(const BCirc* __restrict__ circs, const BEntry* __restrict__ entries, int nteam_entries, int nsingle,
        int nsingle_ctas, int ncirc, const BOp* __restrict__ ops, const typename Ar::coef_t* __restrict__ coefs,
        BCtl* __restrict__ ctl, unsigned int* __restrict__ bars, unsigned long long* __restrict__ times) {
  using raw_t = typename Ar::raw_t;
  using coef_t = typename Ar::coef_t;
  extern __shared__ __align__(16) unsigned char smem[];
  raw_t* sstate = reinterpret_cast<raw_t*>(smem);
  coef_t* sM = reinterpret_cast<coef_t*>(smem + kSmemState);
  uint64_t* smoff = reinterpret_cast<uint64_t*>(smem + kSmemState + kMaxD * kMaxD * sizeof(coef_t));
  __shared__ unsigned int s_next;
  __shared__ int s_queue;            // the queue this CTA takes from now: 0 single-CTA, 1 team
  if (threadIdx.x == 0) {
    atomicMin(&times[ncirc], gtimer());   // launch start (earliest CTA)
    s_queue = (int)blockIdx.x < nsingle_ctas ? 0 : 1;
  }
  for (;;) {
    if (threadIdx.x == 0) {
      // the home queue first, then the other one; done when both are empty
      unsigned int e = 0xFFFFFFFFu;
      for (int tries = 0; tries < 2 && e == 0xFFFFFFFFu; tries++) {
        if (s_queue == 0) {
          const unsigned int qv = atomicAdd(&ctl->queue2, 1u);
          if (qv < (unsigned int)nsingle) e = (unsigned int)nteam_entries + qv;
        } else {
          const unsigned int qv = atomicAdd(&ctl->queue, 1u);
          if (qv < (unsigned int)nteam_entries) e = qv;
        }
        if (e == 0xFFFFFFFFu) s_queue ^= 1;
      }
      s_next = e;
    }
    __syncthreads();
    const unsigned int qi = s_next;
    __syncthreads();
    if (qi == 0xFFFFFFFFu) break;
    const BEntry e = entries[qi];
    const BCirc c = circs[e.circ];
    const uint64_t N = 1ull << c.n;
    raw_t* gst = reinterpret_cast<raw_t*>(c.state);
    raw_t* st = c.smem ? sstate : gst;
    const uint32_t T = (uint32_t)c.team, m = e.member;
    const bool arrive = !(ctl->skip_circ == (int)e.circ && ctl->skip_member == (int)m);
    unsigned int* bar = bars + e.circ;
    raw_t zero;
    zero.x = 0; zero.y = 0;
    {
      const uint64_t a0 = N / T * m, a1 = N / T * (m + 1);
      for (uint64_t i = a0 + threadIdx.x; i < a1; i += kBT) st[i] = zero;
    }
    __syncthreads();
    if (threadIdx.x == 0 && m == 0) { raw_t one; one.x = 1; one.y = 0; st[0] = one; }
    bool ok = T == 1 ? true : team_barrier(bar, T, arrive, ctl);
    for (uint32_t o = 0; o < c.nops && ok; o++) {
      const BOp op = ops[c.op0 + o];
      const int D = 1 << op.k;
      __syncthreads();   // previous op done (and its matrix no longer read)
      for (int i = threadIdx.x; i < D * D; i += kBT) sM[i] = coefs[op.coef + i];
      if (threadIdx.x < D) {
        uint64_t off = 0;
        for (int t = 0; t < op.k; t++)
          if ((threadIdx.x >> (op.k - 1 - t)) & 1) off += 1ull << op.tpos[t];
        smoff[threadIdx.x] = off;
      }
      __syncthreads();
      const uint64_t G = 1ull << (c.n - op.nins);
      const uint64_t g0 = G * m / T, g1 = G * (m + 1) / T;
      if (c.smem) {
        switch (op.k) {
          case 1: apply_op<Ar, 1, false>(st, op, sM, smoff, g0, g1); break;
          case 2: apply_op<Ar, 2, false>(st, op, sM, smoff, g0, g1); break;
          case 3: apply_op<Ar, 3, false>(st, op, sM, smoff, g0, g1); break;
          default: apply_op<Ar, 4, false>(st, op, sM, smoff, g0, g1); break;
        }
      } else {
        switch (op.k) {
          case 1: apply_op<Ar, 1, true>(st, op, sM, smoff, g0, g1); break;
          case 2: apply_op<Ar, 2, true>(st, op, sM, smoff, g0, g1); break;
          case 3: apply_op<Ar, 3, true>(st, op, sM, smoff, g0, g1); break;
          default: apply_op<Ar, 4, true>(st, op, sM, smoff, g0, g1); break;
        }
      }
      if (T > 1) ok = team_barrier(bar, T * (o + 2), arrive, ctl);
    }
    __syncthreads();
    if (c.smem)
      for (uint64_t i = threadIdx.x; i < N; i += kBT) gst[i] = sstate[i];
    __syncthreads();
    if (threadIdx.x == 0 && m == 0) {
      __threadfence();
      times[e.circ] = gtimer();
    }
  }
}

}  // namespace

struct qc_batch {
  int ncirc = 0;
  int dtype = QC_C64, arith = QC_ARITH_AUTO, device = 0;
  int fuse_k = 0, nops = 0, nsmem = 0, team_mb = 8;
  cudaStream_t stream = nullptr;
  void* dmem = nullptr;        // [circs][entries][ops][coefs][ctl][bars][times]
  BCirc* dcircs = nullptr;
  BEntry* dentries = nullptr;
  int nentries = 0;
  BOp* dops = nullptr;
  void* dcoefs = nullptr;
  BCtl* dctl = nullptr;
  int nteam_entries = 0;       // entries [0, nteam_entries): teams of 2..16 CTAs, largest work first
  int nsingle = 0;             // entries after them: single-CTA circuits, smallest work first
  int nsingle_ctas = 0;        // CTAs that start on the single-CTA queue
  unsigned int* dbars = nullptr;
  unsigned long long* dtimes = nullptr;
  BCtl hctl;
  int grid = 1;
  size_t smem = 0;
  cudaGraphExec_t gexec = nullptr;
  std::vector<unsigned long long> htimes;
};

namespace {

template <class Ar>
int build_tables(qc_batch* b, qc_state* const* states, const qc_circuit_desc* circs, int ncirc, int fuse_k,
                 int team_mb) {
  using coef_t = typename Ar::coef_t;
  std::vector<BCirc> hc(ncirc);
  std::vector<BOp> hops;
  std::vector<coef_t> hcoef;
  std::vector<double> work(ncirc);
  b->nsmem = 0;
  for (int i = 0; i < ncirc; i++) {
    const qc_circuit_desc& d = circs[i];
    std::vector<qc_op> ops;
    if (int rc = qc_plan_ops(d.n, d.gates, d.ngates, fuse_k, ops)) return qc_fail(rc, "circuit %d: %s", i, qc_last_error());
    hc[i].state = (uint64_t)(uintptr_t)states[i]->ptr;
    hc[i].n = d.n;
    hc[i].op0 = (uint32_t)hops.size();
    hc[i].nops = (uint32_t)ops.size();
    hc[i].smem = ((size_t)1 << d.n) * sizeof(typename Ar::raw_t) <= kSmemState ? 1 : 0;
    b->nsmem += hc[i].smem;
    for (const qc_op& op : ops) {
      if (op.k > kMaxK) return qc_fail(QC_ERR_UNSUPPORTED, "circuit %d: gate on %d targets (batch path: <= %d)", i, op.k, kMaxK);
      BOp bo;
      std::memset(&bo, 0, sizeof(bo));
      bo.coef = (uint32_t)hcoef.size();
      bo.k = (uint8_t)op.k;
      int ins[QC_MAX_INS], ni = 0;
      for (int t = 0; t < op.k; t++) { bo.tpos[t] = (uint8_t)op.tpos[t]; ins[ni++] = op.tpos[t]; }
      for (int t = 0; t < op.nc; t++) { ins[ni++] = op.cpos[t]; if (op.cval[t]) bo.orval |= 1ull << op.cpos[t]; }
      std::sort(ins, ins + ni);
      bo.nins = (uint8_t)ni;
      for (int t = 0; t < ni; t++) bo.ins[t] = (uint8_t)ins[t];
      const int D = 1 << op.k;
      for (int e = 0; e < D * D; e++) hcoef.push_back(Ar::make_coef(op.U[2 * e], op.U[2 * e + 1]));
      hops.push_back(bo);
    }
    // team size: one CTA per team_mb MB of state beyond shared memory, at most 16
    if (hc[i].smem) {
      hc[i].team = 1;
    } else {
      const size_t bytes = ((size_t)1 << d.n) * sizeof(typename Ar::raw_t);
      int T = 1;
      while (T < 16 && bytes / (size_t)T > ((size_t)team_mb << 20)) T *= 2;
      hc[i].team = T;
    }
    // work per member: sweeps over the state; shared-memory circuits cost a few times less per op
    work[i] = (double)((size_t)1 << d.n) * (double)(ops.size() + 1) * (hc[i].smem ? 0.25 : 1.0) / hc[i].team;
  }
  // Two queues.  Teams (2..16 CTAs), largest work per member first, their
  // entries consecutive (this order bounds the makespan); single-CTA circuits,
  // smallest work first (early completions).  A share of the CTAs
  // proportional to the single-CTA work starts on the second queue; a CTA
  // whose queue is empty moves to the other one.
  std::vector<uint32_t> order(ncirc);
  std::iota(order.begin(), order.end(), 0u);
  std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t c) { return work[a] > work[c]; });
  std::vector<BEntry> ents;
  double wteam = 0.0, wsingle = 0.0;
  for (uint32_t ci : order)
    if (hc[ci].team > 1) {
      for (int m = 0; m < hc[ci].team; m++) ents.push_back(BEntry{ci, (uint32_t)m});
      wteam += work[ci] * hc[ci].team;
    }
  b->nteam_entries = (int)ents.size();
  for (auto it = order.rbegin(); it != order.rend(); ++it)
    if (hc[*it].team == 1) { ents.push_back(BEntry{*it, 0u}); wsingle += work[*it]; }
  b->nsingle = (int)ents.size() - b->nteam_entries;
  const size_t sz_c = sizeof(BCirc) * ncirc, sz_e = (sizeof(BEntry) * ents.size() + 15) & ~(size_t)15;
  const size_t sz_op = sizeof(BOp) * std::max<size_t>(1, hops.size());
  const size_t sz_cf = (sizeof(coef_t) * std::max<size_t>(1, hcoef.size()) + 15) & ~(size_t)15;
  const size_t sz_ctl = (sizeof(BCtl) + 15) & ~(size_t)15;
  const size_t sz_b = (sizeof(unsigned int) * ncirc + 15) & ~(size_t)15;
  const size_t sz_t = sizeof(unsigned long long) * (ncirc + 1);
  const size_t total = sz_c + sz_e + sz_op + sz_cf + sz_ctl + sz_b + sz_t;
  void* m = nullptr;
  cudaError_t e = cudaMalloc(&m, total);
  if (e != cudaSuccess) { cudaGetLastError(); return qc_fail(QC_ERR_OOM, "batch tables (%zu bytes)", total); }
  if (b->dmem) cudaFree(b->dmem);
  b->dmem = m;
  char* p = (char*)m;
  b->dcircs = (BCirc*)p; p += sz_c;
  b->dentries = (BEntry*)p; p += sz_e;
  b->dops = (BOp*)p; p += sz_op;
  b->dcoefs = p; p += sz_cf;
  b->dctl = (BCtl*)p; p += sz_ctl;
  b->dbars = (unsigned int*)p; p += sz_b;
  b->dtimes = (unsigned long long*)p;
  b->nentries = (int)ents.size();
  QC_CUDA(cudaMemcpy(b->dcircs, hc.data(), sz_c, cudaMemcpyHostToDevice));
  QC_CUDA(cudaMemcpy(b->dentries, ents.data(), sizeof(BEntry) * ents.size(), cudaMemcpyHostToDevice));
  if (!hops.empty()) QC_CUDA(cudaMemcpy(b->dops, hops.data(), sizeof(BOp) * hops.size(), cudaMemcpyHostToDevice));
  if (!hcoef.empty()) QC_CUDA(cudaMemcpy(b->dcoefs, hcoef.data(), sizeof(coef_t) * hcoef.size(), cudaMemcpyHostToDevice));
  b->nops = (int)hops.size();
  b->fuse_k = fuse_k;
  b->smem = kSmemState + kMaxD * kMaxD * sizeof(coef_t) + kMaxD * sizeof(uint64_t);
  QC_CUDA(cudaFuncSetAttribute(k_batch<Ar>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem));
  QC_CUDA(cudaFuncSetAttribute(k_batch<Ar>, cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared));
  int per_sm = 0;
  QC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<Ar>, kBT, b->smem));
  // never more CTAs than can be resident at once: team barriers rely on it
  b->grid = std::max(1, std::min(b->nentries, qc_num_sms() * std::max(1, per_sm)));
  if (b->grid < 16 && b->nentries > b->grid) return qc_fail(QC_ERR_UNSUPPORTED, "device too small for batch teams");
  // CTAs starting on the single-CTA queue: their share of the work, leaving at least 16 for the teams
  int ns = (int)((double)b->grid * wsingle / std::max(1e-30, wteam + wsingle) + 0.5);
  if (b->nsingle > 0) ns = std::max(ns, 1);
  if (b->nteam_entries > 0) ns = std::min(ns, b->grid - 16);
  b->nsingle_ctas = std::max(0, ns);
  return QC_OK;
}

template <class Ar>
int enqueue(qc_batch* b) {
  QC_CUDA(cudaMemcpyAsync(b->dctl, &b->hctl, sizeof(BCtl), cudaMemcpyHostToDevice, b->stream));
  QC_CUDA(cudaMemsetAsync(b->dbars, 0, sizeof(unsigned int) * b->ncirc, b->stream));
  QC_CUDA(cudaMemsetAsync(b->dtimes + b->ncirc, 0xFF, sizeof(unsigned long long), b->stream));
  k_batch<Ar><<<b->grid, kBT, b->smem, b->stream>>>(b->dcircs, b->dentries, b->nteam_entries, b->nsingle,
                                                   b->nsingle_ctas, b->ncirc, b->dops,
                                                   (const typename Ar::coef_t*)b->dcoefs, b->dctl, b->dbars,
                                                   b->dtimes);
  QC_LAUNCHED("k_batch");
  return QC_OK;
}

int read_status(qc_batch* b) {
  int st = 0;
  QC_CUDA(cudaMemcpy(&st, &b->dctl->status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st) return qc_fail(QC_ERR_TIMEOUT, "a team barrier of the batch kernel gave up; results are incomplete");
  return QC_OK;
}

int enqueue_any(qc_batch* b) {
  if (b->dtype == QC_C64) return enqueue<ArC64>(b);
  if (b->arith == QC_ARITH_NATIVE) return enqueue<ArC128>(b);
  return enqueue<ArC128x>(b);
}

int build_any(qc_batch* b, qc_state* const* states, const qc_circuit_desc* circs, int ncirc, int fuse_k,
              int team_mb) {
  if (b->dtype == QC_C64) return build_tables<ArC64>(b, states, circs, ncirc, fuse_k, team_mb);
  if (b->arith == QC_ARITH_NATIVE) return build_tables<ArC128>(b, states, circs, ncirc, fuse_k, team_mb);
  return build_tables<ArC128x>(b, states, circs, ncirc, fuse_k, team_mb);
}

int timed_run(qc_batch* b, float* ms) {
  cudaEvent_t e0, e1;
  QC_CUDA(cudaEventCreate(&e0));
  QC_CUDA(cudaEventCreate(&e1));
  cudaEventRecord(e0, b->stream);
  int rc = enqueue_any(b);
  cudaEventRecord(e1, b->stream);
  if (rc == QC_OK) {
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) rc = qc_cuda_fail(e, "batch run");
    else cudaEventElapsedTime(ms, e0, e1);
  }
  if (rc == QC_OK) rc = read_status(b);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

}  // namespace

extern "C" int qc_batch_create(qc_state* const* states, const qc_circuit_desc* circs, int ncirc,
                               const qc_batch_opts* opts, qc_batch** out) {
  if (!out) return qc_fail(QC_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (ncirc < 1 || !states || !circs) return qc_fail(QC_ERR_ARG, "empty or NULL batch");
  qc_batch_opts o;
  std::memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  if (o.fuse_k > kMaxK) return qc_fail(QC_ERR_ARG, "fuse_k=%d (batch path supports up to %d)", o.fuse_k, kMaxK);
  for (int i = 0; i < ncirc; i++) {
    if (int rc = qc_check_state(states[i])) return qc_fail(rc, "state %d: %s", i, qc_last_error());
    if (states[i]->n != circs[i].n) return qc_fail(QC_ERR_ARG, "state %d has n=%d, circuit has n=%d", i, states[i]->n, circs[i].n);
    if (states[i]->dtype != states[0]->dtype || states[i]->arith != states[0]->arith || states[i]->device != states[0]->device)
      return qc_fail(QC_ERR_ARG, "state %d: all states of a batch need one dtype, arith and device", i);
    if (circs[i].ngates < 0 || (circs[i].ngates > 0 && !circs[i].gates)) return qc_fail(QC_ERR_ARG, "circuit %d: invalid gate list", i);
  }
  qc_batch* b = new qc_batch;
  b->ncirc = ncirc;
  b->dtype = states[0]->dtype;
  b->arith = states[0]->arith;
  b->device = states[0]->device;
  b->stream = (cudaStream_t)o.stream;
  b->htimes.resize(ncirc + 1);
  std::memset(&b->hctl, 0, sizeof(b->hctl));
  b->hctl.skip_circ = o.test_skip_circuit > 0 ? o.test_skip_circuit - 1 : -1;
  b->hctl.skip_member = o.test_skip_member;
  b->hctl.spin_limit = o.spin_limit > 0 ? (unsigned long long)o.spin_limit : (1ull << 26);
  int rc = QC_OK;
  if (o.fuse_k < 0) {
    // autotune: time the whole batch once per candidate (fusion width, state
    // bytes per team member), keep the fastest
    float best = 1e30f;
    int bestk = 1, bestmb = 8;
    for (int k : {2, 3, 4}) {
      for (int mb : {4, 8, 16}) {
        rc = build_any(b, states, circs, ncirc, k, mb);
        float ms = 0.f;
        if (rc == QC_OK) rc = timed_run(b, &ms);
        if (rc != QC_OK) break;
        if (ms < best) { best = ms; bestk = k; bestmb = mb; }
      }
      if (rc != QC_OK) break;
    }
    b->team_mb = bestmb;
    if (rc == QC_OK) rc = build_any(b, states, circs, ncirc, bestk, bestmb);
  } else {
    b->team_mb = 8;
    rc = build_any(b, states, circs, ncirc, o.fuse_k, 8);
  }
  if (rc == QC_OK && o.use_graph) {
    if (!b->stream) rc = qc_fail(QC_ERR_ARG, "graph capture needs a non-default stream");
    cudaGraph_t g = nullptr;
    if (rc == QC_OK) {
      cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) rc = qc_cuda_fail(e, "cudaStreamBeginCapture");
    }
    if (rc == QC_OK) {
      int rc2 = enqueue_any(b);
      cudaError_t e = cudaStreamEndCapture(b->stream, &g);
      if (rc2 != QC_OK) rc = rc2;
      else if (e != cudaSuccess) rc = qc_cuda_fail(e, "cudaStreamEndCapture");
    }
    if (rc == QC_OK) {
      cudaError_t e = cudaGraphInstantiate(&b->gexec, g, 0);
      if (e != cudaSuccess) rc = qc_cuda_fail(e, "cudaGraphInstantiate");
    }
    if (g) cudaGraphDestroy(g);
  }
  if (rc != QC_OK) {
    qc_batch_free(b);
    return rc;
  }
  *out = b;
  return QC_OK;
}

extern "C" int qc_batch_launch(qc_batch* b, double* completion_ms, double* total_ms) {
  if (!b) return qc_fail(QC_ERR_ARG, "batch is NULL");
  QC_CUDA(cudaSetDevice(b->device));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (total_ms) {
    QC_CUDA(cudaEventCreate(&e0));
    QC_CUDA(cudaEventCreate(&e1));
    cudaEventRecord(e0, b->stream);
  }
  int rc = QC_OK;
  if (b->gexec) {
    cudaError_t e = cudaGraphLaunch(b->gexec, b->stream);
    if (e != cudaSuccess) rc = qc_cuda_fail(e, "cudaGraphLaunch");
  } else {
    rc = enqueue_any(b);
  }
  if (total_ms) cudaEventRecord(e1, b->stream);
  if (rc == QC_OK && (completion_ms || total_ms)) {
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) rc = qc_cuda_fail(e, "batch run");
    if (rc == QC_OK) rc = read_status(b);
    if (rc == QC_OK && completion_ms) {
      e = cudaMemcpy(b->htimes.data(), b->dtimes, sizeof(unsigned long long) * (b->ncirc + 1), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) rc = qc_cuda_fail(e, "cudaMemcpy(times)");
      const unsigned long long t0 = b->htimes[b->ncirc];
      for (int i = 0; i < b->ncirc && rc == QC_OK; i++) completion_ms[i] = (double)(b->htimes[i] - t0) * 1e-6;
    }
    if (rc == QC_OK && total_ms) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      *total_ms = ms;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return rc;
}

extern "C" int qc_batch_info(const qc_batch* b, int* fuse_k, int* nops, int* nsmem) {
  if (!b) return qc_fail(QC_ERR_ARG, "batch is NULL");
  if (fuse_k) *fuse_k = b->fuse_k;
  if (nops) *nops = b->nops;
  if (nsmem) *nsmem = b->nsmem;
  return QC_OK;
}

extern "C" int qc_batch_free(qc_batch* b) {
  if (!b) return QC_OK;
  cudaSetDevice(b->device);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->dmem) cudaFree(b->dmem);
  delete b;
  return QC_OK;
}
