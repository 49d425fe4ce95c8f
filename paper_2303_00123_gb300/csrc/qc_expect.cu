// qc_expect.cu -- <psi| sum_t c_t P_t |psi> for Pauli sums, FP64 reductions.
//
// For a Pauli string P with flip mask F (its X and Y qubits), phase mask
// Q (its Y and Z qubits) and nY Y factors, P|y> = i^nY (-1)^popc(y & Q) |y^F>
// (X|b> = |1-b>, Y|b> = i(-1)^b |1-b>, Z|b> = (-1)^b |b>), so
//   <psi|P|psi> = sum_y i^nY (-1)^popc(y & Q) conj(psi_{y^F}) psi_y .
// Terms that share F are evaluated in one sweep: the kernel visits each pair
// {y, y^F} once (y with the pivot bit of F clear), forms the overlap products
// and adds every term's signed contribution to an FP64 accumulator.  Per-block
// partial sums go to device scratch memory; a single-block kernel adds them up
// in a fixed order, so the result is deterministic.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "qc_common.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxTermsPerSweep = 64;

struct TermSet {
  uint64_t flip;                 // F (bit positions)
  int pivot;                     // a set bit of F (or -1 when F == 0)
  int nterms;
  uint64_t phase_mask[kMaxTermsPerSweep];
  double coeff[kMaxTermsPerSweep];   // c_t * Re/Im selector folded in below
  int ipow[kMaxTermsPerSweep];       // nY mod 4
};

// Amplitude loads in FP64 (complex64 is widened; FP64 arithmetic follows).
__device__ __forceinline__ double2 ld_amp(const float2* p, uint64_t i) { float2 v = p[i]; return make_double2(v.x, v.y); }
__device__ __forceinline__ double2 ld_amp(const double2* p, uint64_t i) { return p[i]; }

// Re(i^k * z)
__device__ __forceinline__ double re_ipow(int k, double2 z) {
  switch (k & 3) {
    case 0: return z.x;
    case 1: return -z.y;
    case 2: return -z.x;
    default: return z.y;
  }
}

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < kThreads / 32 ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  __syncthreads();
  return t;
}

template <class T>
__global__ void __launch_bounds__(kThreads)
k_pauli_sweep(const T* __restrict__ psi, uint64_t npairs, const __grid_constant__ TermSet ts, double* __restrict__ partial) {
  double acc = 0.0;
  const uint64_t stride = (uint64_t)gridDim.x * kThreads;
  for (uint64_t j = (uint64_t)blockIdx.x * kThreads + threadIdx.x; j < npairs; j += stride) {
    if (ts.pivot < 0) {
      // diagonal terms: sum_y |psi_y|^2 (-1)^popc(y & Q)
      const double2 a = ld_amp(psi, j);
      const double p = a.x * a.x + a.y * a.y;
      double s = 0.0;
      for (int t = 0; t < ts.nterms; t++) {
        const double sg = (__popcll(j & ts.phase_mask[t]) & 1) ? -1.0 : 1.0;
        s += sg * ts.coeff[t];   // diagonal strings contain no Y: i^nY = 1
      }
      acc += s * p;
    } else {
      const uint64_t y = qc_insert_zero(j, ts.pivot);
      const uint64_t z = y ^ ts.flip;
      const double2 a = ld_amp(psi, y), b = ld_amp(psi, z);
      // w = conj(psi_z) psi_y  (contribution of y);  conj(w) (contribution of z)
      const double2 w = make_double2(b.x * a.x + b.y * a.y, b.x * a.y - b.y * a.x);
      const double2 wc = make_double2(w.x, -w.y);
      double s = 0.0;
      for (int t = 0; t < ts.nterms; t++) {
        const double sy = (__popcll(y & ts.phase_mask[t]) & 1) ? -1.0 : 1.0;
        const double sz = (__popcll(z & ts.phase_mask[t]) & 1) ? -1.0 : 1.0;
        s += ts.coeff[t] * (sy * re_ipow(ts.ipow[t], w) + sz * re_ipow(ts.ipow[t], wc));
      }
      acc += s;
    }
  }
  const double tot = block_sum(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

__global__ void k_sum_partials(const double* __restrict__ partial, int n, double* __restrict__ out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += kThreads) acc += partial[i];
  const double t = block_sum(acc);
  if (threadIdx.x == 0) out[0] = t;
}

// Grow-only device scratch buffer per device (partials + result).
std::mutex g_scratch_mu;
std::map<int, std::pair<void*, size_t>> g_scratch;

// Callers hold g_scratch_mu for the whole call (qc_expect is synchronous), so
// concurrent calls from several host threads do not share the buffer in flight.
int get_scratch(int device, size_t bytes, void** p) {
  auto& e = g_scratch[device];
  if (e.second < bytes) {
    if (e.first) cudaFree(e.first);
    e.first = nullptr;
    e.second = 0;
    cudaError_t err = cudaMalloc(&e.first, bytes);
    if (err != cudaSuccess) { e.first = nullptr; return qc_cuda_fail(err, "cudaMalloc(scratch)"); }
    e.second = bytes;
  }
  *p = e.first;
  return QC_OK;
}

}  // namespace

namespace {
// Parse a Pauli sum into sweeps (one TermSet per distinct flip mask; identity
// factors are dropped, an all-identity term is a diagonal term with Q = 0).
int pauli_plan(int n, const qc_pauli_sum* H, std::vector<TermSet>& sets) {
  if (!H || H->nterms < 0) return qc_fail(QC_ERR_ARG, "invalid Pauli sum");
  if (H->nterms > 0 && (!H->coeffs || !H->offsets)) return qc_fail(QC_ERR_ARG, "Pauli sum arrays are NULL");
  std::map<uint64_t, size_t> by_flip;
  for (int t = 0; t < H->nterms; t++) {
    const int b = H->offsets[t], e = H->offsets[t + 1];
    if (e < b) return qc_fail(QC_ERR_ARG, "term %d: offsets decrease", t);
    if (e > b && (!H->letters || !H->qubits)) return qc_fail(QC_ERR_ARG, "Pauli letters/qubits are NULL");
    uint64_t F = 0, Q = 0, used = 0;
    int ny = 0;
    for (int i = b; i < e; i++) {
      const int q = H->qubits[i];
      if (q < 0 || q >= n) return qc_fail(QC_ERR_ARG, "term %d: qubit %d out of range", t, q);
      const uint64_t bit = 1ull << (n - 1 - q);
      const char L = H->letters[i];
      if (L == 'I' || L == 'i') continue;
      if (used & bit) return qc_fail(QC_ERR_ARG, "term %d: qubit %d appears twice", t, q);
      used |= bit;
      if (L == 'X' || L == 'x') F |= bit;
      else if (L == 'Y' || L == 'y') { F |= bit; Q |= bit; ny++; }
      else if (L == 'Z' || L == 'z') Q |= bit;
      else return qc_fail(QC_ERR_ARG, "term %d: unknown Pauli letter '%c'", t, L);
    }
    const double c = H->coeffs[t];
    auto it = by_flip.find(F);
    if (it == by_flip.end() || sets[it->second].nterms == kMaxTermsPerSweep) {
      TermSet ts;
      std::memset(&ts, 0, sizeof(ts));
      ts.flip = F;
      ts.pivot = F ? 63 - __builtin_clzll(F) : -1;
      by_flip[F] = sets.size();
      sets.push_back(ts);
      it = by_flip.find(F);
    }
    TermSet& ts = sets[it->second];
    ts.phase_mask[ts.nterms] = Q;
    ts.coeff[ts.nterms] = c;
    ts.ipow[ts.nterms] = ny & 3;
    ts.nterms++;
  }
  return QC_OK;
}
}  // namespace

extern "C" int qc_expect(const qc_state* s, const qc_pauli_sum* H, double* out) {
  if (int rc = qc_check_state(s)) return rc;
  if (!out) return qc_fail(QC_ERR_ARG, "out is NULL");
  std::vector<TermSet> sets;
  if (int rc = pauli_plan(s->n, H, sets)) return rc;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  const uint64_t N = 1ull << s->n;
  const int cap = qc_num_sms() * 8;
  // grid per sweep and scratch layout: [partials of sweep 0 | sweep 1 | ...][result]
  std::vector<int> grids(sets.size());
  size_t total = 0;
  for (size_t i = 0; i < sets.size(); i++) {
    const uint64_t npairs = sets[i].pivot < 0 ? N : N / 2;
    grids[i] = (int)std::max<uint64_t>(1, std::min<uint64_t>((npairs + kThreads - 1) / kThreads, cap));
    total += grids[i];
  }
  void* scratch = nullptr;
  if (int rc = get_scratch(s->device, (total + 1) * sizeof(double), &scratch)) return rc;
  double* partial = (double*)scratch;
  size_t off = 0;
  for (size_t i = 0; i < sets.size(); i++) {
    const uint64_t npairs = sets[i].pivot < 0 ? N : N / 2;
    if (s->dtype == QC_C64)
      k_pauli_sweep<float2><<<grids[i], kThreads, 0, s->stream>>>((const float2*)s->ptr, npairs, sets[i], partial + off);
    else
      k_pauli_sweep<double2><<<grids[i], kThreads, 0, s->stream>>>((const double2*)s->ptr, npairs, sets[i], partial + off);
    QC_LAUNCHED("k_pauli_sweep");
    off += grids[i];
  }
  double result = 0.0;
  if (total > 0) {
    k_sum_partials<<<1, kThreads, 0, s->stream>>>(partial, (int)total, partial + total);
    QC_LAUNCHED("k_sum_partials");
    QC_CUDA(cudaMemcpyAsync(&result, partial + total, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  }
  QC_CUDA(cudaStreamSynchronize(s->stream));
  *out = result;
  return QC_OK;
}

// ---------------------------------------------------------------------------
// qc_expect_noalloc: the same sweeps and reductions as qc_expect, with the
// partial sums held in a fixed device array instead of a heap buffer.
// Layout of the array: [kNaPartials partials of the current sweep]
// [kNaSweeps per-sweep sums][1 final sum].  Each call writes every slot it
// later reads, so nothing has to be cleared between calls.
namespace {
constexpr int kNaPartials = 4096;   // blocks per sweep (grid is capped at this)
constexpr int kNaSweeps = 1023;     // distinct X/Y patterns (64 terms per sweep)
static __device__ __align__(256) double g_na_scratch[kNaPartials + kNaSweeps + 1];

std::mutex g_na_mu;
double* g_na_ptr[64] = {nullptr};   // device address of g_na_scratch, per device

int na_setup(int dev, double** p) {
  if (dev < 0 || dev >= 64) return qc_fail(QC_ERR_UNSUPPORTED, "device ordinal %d >= 64", dev);
  if (!g_na_ptr[dev]) {
    void* a = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&a, g_na_scratch);   // the state's device is current
    if (e != cudaSuccess) return qc_cuda_fail(e, "cudaGetSymbolAddress(g_na_scratch)");
    g_na_ptr[dev] = (double*)a;
  }
  *p = g_na_ptr[dev];
  return QC_OK;
}

// Flip and phase masks of term t (validated); returns QC_OK or an error.
int na_term(int n, const qc_pauli_sum* H, int t, uint64_t* F, uint64_t* Q, int* ny) {
  const int b = H->offsets[t], e = H->offsets[t + 1];
  if (e < b) return qc_fail(QC_ERR_ARG, "term %d: offsets decrease", t);
  if (e > b && (!H->letters || !H->qubits)) return qc_fail(QC_ERR_ARG, "Pauli letters/qubits are NULL");
  uint64_t f = 0, q = 0, used = 0;
  int y = 0;
  for (int i = b; i < e; i++) {
    const int qb = H->qubits[i];
    if (qb < 0 || qb >= n) return qc_fail(QC_ERR_ARG, "term %d: qubit %d out of range", t, qb);
    const uint64_t bit = 1ull << (n - 1 - qb);
    const char L = H->letters[i];
    if (L == 'I' || L == 'i') continue;
    if (used & bit) return qc_fail(QC_ERR_ARG, "term %d: qubit %d appears twice", t, qb);
    used |= bit;
    if (L == 'X' || L == 'x') f |= bit;
    else if (L == 'Y' || L == 'y') { f |= bit; q |= bit; y++; }
    else if (L == 'Z' || L == 'z') q |= bit;
    else return qc_fail(QC_ERR_ARG, "term %d: unknown Pauli letter '%c'", t, L);
  }
  *F = f;
  *Q = q;
  *ny = y;
  return QC_OK;
}
}  // namespace

extern "C" int qc_expect_noalloc(const qc_state* s, const qc_pauli_sum* H, double* out) {
  if (int rc = qc_check_state(s)) return rc;
  if (!out) return qc_fail(QC_ERR_ARG, "out is NULL");
  if (!H || H->nterms < 0) return qc_fail(QC_ERR_ARG, "invalid Pauli sum");
  if (H->nterms > 0 && (!H->coeffs || !H->offsets)) return qc_fail(QC_ERR_ARG, "Pauli sum arrays are NULL");
  // Validate every term and count the sweeps before touching the device.
  int nsweeps = 0;
  for (int t = 0; t < H->nterms; t++) {
    uint64_t F, Q;
    int ny;
    if (int rc = na_term(s->n, H, t, &F, &Q, &ny)) return rc;
    bool seen = false;
    for (int u = 0; u < t && !seen; u++) {
      uint64_t F2, Q2;
      int ny2;
      na_term(s->n, H, u, &F2, &Q2, &ny2);
      seen = (F2 == F);
    }
    if (seen) continue;
    int cnt = 0;
    for (int u = t; u < H->nterms; u++) {
      uint64_t F2, Q2;
      int ny2;
      na_term(s->n, H, u, &F2, &Q2, &ny2);
      if (F2 == F) cnt++;
    }
    nsweeps += (cnt + kMaxTermsPerSweep - 1) / kMaxTermsPerSweep;
  }
  if (nsweeps > kNaSweeps)
    return qc_fail(QC_ERR_ARG, "qc_expect_noalloc: %d sweeps needed, the fixed scratch holds at most %d "
                   "(distinct X/Y patterns, 64 terms per sweep)", nsweeps, kNaSweeps);
  std::lock_guard<std::mutex> lk(g_na_mu);
  double* scratch = nullptr;
  if (int rc = na_setup(s->device, &scratch)) return rc;
  double* partial = scratch;
  double* sweep_sum = scratch + kNaPartials;
  double* final_sum = sweep_sum + kNaSweeps;
  const uint64_t N = 1ull << s->n;
  const int cap = std::min(qc_num_sms() * 8, kNaPartials);
  int sw = 0;
  for (int t = 0; t < H->nterms; t++) {
    uint64_t F, Q;
    int ny;
    na_term(s->n, H, t, &F, &Q, &ny);
    bool seen = false;
    for (int u = 0; u < t && !seen; u++) {
      uint64_t F2, Q2;
      int ny2;
      na_term(s->n, H, u, &F2, &Q2, &ny2);
      seen = (F2 == F);
    }
    if (seen) continue;
    TermSet ts;
    std::memset(&ts, 0, sizeof(ts));
    ts.flip = F;
    ts.pivot = F ? 63 - __builtin_clzll(F) : -1;
    const uint64_t npairs = F ? N / 2 : N;
    const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((npairs + kThreads - 1) / kThreads, cap));
    for (int u = t; u <= H->nterms; u++) {
      bool flush = (u == H->nterms);
      if (!flush) {
        uint64_t F2, Q2;
        int ny2;
        na_term(s->n, H, u, &F2, &Q2, &ny2);
        if (F2 != F) continue;
        ts.phase_mask[ts.nterms] = Q2;
        ts.coeff[ts.nterms] = H->coeffs[u];
        ts.ipow[ts.nterms] = ny2 & 3;
        ts.nterms++;
        flush = (ts.nterms == kMaxTermsPerSweep);
      }
      if (flush && ts.nterms > 0) {
        if (s->dtype == QC_C64)
          k_pauli_sweep<float2><<<grid, kThreads, 0, s->stream>>>((const float2*)s->ptr, npairs, ts, partial);
        else
          k_pauli_sweep<double2><<<grid, kThreads, 0, s->stream>>>((const double2*)s->ptr, npairs, ts, partial);
        k_sum_partials<<<1, kThreads, 0, s->stream>>>(partial, grid, sweep_sum + sw);
        QC_LAUNCHED("qc_expect_noalloc sweep");
        sw++;
        ts.nterms = 0;
      }
    }
  }
  double result = 0.0;
  if (sw > 0) {
    k_sum_partials<<<1, kThreads, 0, s->stream>>>(sweep_sum, sw, final_sum);
    QC_LAUNCHED("qc_expect_noalloc final sum");
    QC_CUDA(cudaMemcpyAsync(&result, final_sum, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  }
  QC_CUDA(cudaStreamSynchronize(s->stream));
  *out = result;
  return QC_OK;
}
