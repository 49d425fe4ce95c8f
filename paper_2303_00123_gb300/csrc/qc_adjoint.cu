// qc_adjoint.cu -- batched adjoint (reverse-sweep) gradients.
//
// For |psi> = U_L ... U_1 |0> and E = <psi|H|psi>, with parametric gates
// U_l = exp(-i theta_l P_l / 2), dU_l/dtheta_l = -(i/2) P_l U_l, so
//   dE/dtheta_l = 2 Re <lambda_l| dU_l/dtheta |phi_{l-1}> = Im <lambda_l| P_l |phi_l>
// with phi_l = U_l ... U_1 |0> and lambda_l = U_{l+1}^dag ... U_L^dag H |psi>
// (Jones & Gacon 2020, arXiv:2009.02823).  One forward sweep builds phi_L =
// psi, one gather kernel forms lambda_L = H psi, then the circuit is walked
// backwards: at a parametric gate the kernel reduces Im <lambda|P|phi> over
// the gate's qubit pairs and, in the same pass over the same pairs, undoes the
// gate on phi and on lambda.  Only the two states per parameter set are kept.
//
// Layout: a workspace of 2*B states, phi_b at [b], lambda_b at [B + b]; every
// kernel runs over (groups, states) with the state index in blockIdx.y.  Gate
// matrices for all gates (and all parameter sets, for the parametric ones) are
// uploaded once per call.  Reductions accumulate in FP64: per-block partial
// sums, then one block per parameter set adds them in a fixed order.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "qc_common.cuh"

namespace {

constexpr int kT = 256;
constexpr int kMaxHTerms = 256;

struct HTerms {
  int nterms;
  uint64_t flip[kMaxHTerms];
  uint64_t phase[kMaxHTerms];
  double coeff[kMaxHTerms];
  int ipow[kMaxHTerms];
};

template <class R> struct Cx;
template <> struct Cx<float> { using t = float2; };
template <> struct Cx<double> { using t = double2; };

template <class Ar> struct RedT;
template <> struct RedT<ArC64> { using R = float; };
template <> struct RedT<ArC128> { using R = double; };
template <> struct RedT<ArC128x> { using R = double; };

__device__ __forceinline__ double block_sum_d(double v) {
  __shared__ double red[kT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < kT / 32 ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  __syncthreads();
  return t;
}

// Block sum in the state's precision class: complex64 states reduce in FP32
// within a block (256 products of FP32 values; GB300's FP64 pipe runs at a
// small fraction of the FP32 rate), complex128 in FP64; block totals are
// summed across blocks in FP64.
__device__ __forceinline__ float block_sum_f(float v) {
  __shared__ float redf[kT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) redf[threadIdx.x >> 5] = v;
  __syncthreads();
  float t = 0.f;
  if (threadIdx.x < 32) {
    t = threadIdx.x < kT / 32 ? redf[threadIdx.x] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  __syncthreads();
  return t;
}
__device__ __forceinline__ double block_sum_r(float v) { return (double)block_sum_f(v); }
__device__ __forceinline__ double block_sum_r(double v) { return block_sum_d(v); }

// ---------------------------------------------------------------- gates
struct BGeom {
  uint64_t ngroups;       // groups per state
  uint64_t nstate;        // amplitudes per state
  uint64_t orval;
  uint64_t moff[4];       // member offsets (K <= 2)
  int nins;
  int ins[QC_MAX_INS];
  int B;                  // parameter sets; matrix of state s is mats[(s % B) * mstride]
  int mstride;            // coef_t entries between consecutive parameter sets (0: shared)
};

template <class Ar, int K>
__global__ void __launch_bounds__(kT)
k_bgate(typename Ar::raw_t* __restrict__ base, const __grid_constant__ BGeom g,
        const typename Ar::coef_t* __restrict__ mats) {
  constexpr int D = 1 << K;
  __shared__ typename Ar::coef_t M[D * D];
  const int s = blockIdx.y;
  const typename Ar::coef_t* m = mats + (size_t)(s % g.B) * g.mstride;
  if (threadIdx.x < D * D) M[threadIdx.x] = m[threadIdx.x];
  __syncthreads();
  typename Ar::raw_t* st = base + (size_t)s * g.nstate;
  for (uint64_t j = (uint64_t)blockIdx.x * kT + threadIdx.x; j < g.ngroups; j += (uint64_t)gridDim.x * kT) {
    uint64_t b = j;
    for (int i = 0; i < g.nins; i++) b = qc_insert_zero(b, g.ins[i]);
    b |= g.orval;
    typename Ar::val_t in[D];
#pragma unroll
    for (int r = 0; r < D; r++) in[r] = Ar::from_raw(st[b + g.moff[r]]);
#pragma unroll
    for (int r = 0; r < D; r++) st[b + g.moff[r]] = Ar::to_raw(Ar::template dot<D>(&M[r * D], in));
  }
}

// Parametric gate on target position t with generator P (0: X, 1: Y, 2: Z):
// partial[s][block] = sum over pairs of Im<lambda|P|phi>, then both phi and
// lambda are multiplied by the per-set matrix (U^dag) on the same pairs.
template <class Ar>
__global__ void __launch_bounds__(kT)
k_adj_param(typename Ar::raw_t* __restrict__ work, uint64_t nstate, int B, int t, int P,
            const typename Ar::coef_t* __restrict__ mats, double* __restrict__ partial) {
  using R = typename RedT<Ar>::R;
  __shared__ typename Ar::coef_t M[4];
  const int s = blockIdx.y;   // parameter set
  if (threadIdx.x < 4) M[threadIdx.x] = mats[(size_t)s * 4 + threadIdx.x];
  __syncthreads();
  typename Ar::raw_t* phi = work + (size_t)s * nstate;
  typename Ar::raw_t* lam = work + (size_t)(B + s) * nstate;
  const uint64_t npairs = nstate >> 1, off = 1ull << t;
  R acc = 0;
  for (uint64_t j = (uint64_t)blockIdx.x * kT + threadIdx.x; j < npairs; j += (uint64_t)gridDim.x * kT) {
    const uint64_t a = qc_insert_zero(j, t), b = a + off;
    const typename Ar::raw_t pa = phi[a], pb = phi[b], la = lam[a], lb = lam[b];
    const R par = (R)pa.x, pai = (R)pa.y, pbr = (R)pb.x, pbi = (R)pb.y;
    const R lar = (R)la.x, lai = (R)la.y, lbr = (R)lb.x, lbi = (R)lb.y;
    R c;
    if (P == 2) {        // Z: Im(conj(la) pa) - Im(conj(lb) pb)
      c = (lar * pai - lai * par) - (lbr * pbi - lbi * pbr);
    } else if (P == 0) { // X: Im(conj(la) pb) + Im(conj(lb) pa)
      c = (lar * pbi - lai * pbr) + (lbr * pai - lbi * par);
    } else {             // Y: -Re(conj(la) pb) + Re(conj(lb) pa)
      c = -(lar * pbr + lai * pbi) + (lbr * par + lbi * pai);
    }
    acc += c;
    typename Ar::val_t v[2];
    v[0] = Ar::from_raw(pa); v[1] = Ar::from_raw(pb);
    phi[a] = Ar::to_raw(Ar::template dot<2>(&M[0], v));
    phi[b] = Ar::to_raw(Ar::template dot<2>(&M[2], v));
    v[0] = Ar::from_raw(la); v[1] = Ar::from_raw(lb);
    lam[a] = Ar::to_raw(Ar::template dot<2>(&M[0], v));
    lam[b] = Ar::to_raw(Ar::template dot<2>(&M[2], v));
  }
  const double tot = block_sum_r(acc);
  if (threadIdx.x == 0) partial[(size_t)s * gridDim.x + blockIdx.x] = tot;
}

// lambda_s = H phi_s (gather: each output index collects every term).
template <class T>
__global__ void __launch_bounds__(kT)
k_hamiltonian(T* __restrict__ work, uint64_t nstate, int B, const __grid_constant__ HTerms h) {
  using R = decltype(T::x);
  const int s = blockIdx.y;
  const T* phi = work + (size_t)s * nstate;
  T* lam = work + (size_t)(B + s) * nstate;
  for (uint64_t z = (uint64_t)blockIdx.x * kT + threadIdx.x; z < nstate; z += (uint64_t)gridDim.x * kT) {
    R re = 0, im = 0;
    for (int k = 0; k < h.nterms; k++) {
      const uint64_t y = z ^ h.flip[k];
      const T v = phi[y];
      R c = (R)h.coeff[k];
      if (__popcll(y & h.phase[k]) & 1) c = -c;
      switch (h.ipow[k]) {   // c * i^p * v
        case 0: re += c * v.x; im += c * v.y; break;
        case 1: re -= c * v.y; im += c * v.x; break;
        case 2: re -= c * v.x; im -= c * v.y; break;
        default: re += c * v.y; im -= c * v.x; break;
      }
    }
    T o;
    o.x = re;
    o.y = im;
    lam[z] = o;
  }
}

// partial[s][block] = sum Re(conj(phi_s) lambda_s)
template <class T>
__global__ void __launch_bounds__(kT)
k_energy(const T* __restrict__ work, uint64_t nstate, int B, double* __restrict__ partial) {
  const int s = blockIdx.y;
  const T* phi = work + (size_t)s * nstate;
  const T* lam = work + (size_t)(B + s) * nstate;
  using R = decltype(T::x);
  R acc = 0;
  for (uint64_t z = (uint64_t)blockIdx.x * kT + threadIdx.x; z < nstate; z += (uint64_t)gridDim.x * kT) {
    const T a = phi[z], b = lam[z];
    acc += a.x * b.x + a.y * b.y;
  }
  const double tot = block_sum_r(acc);
  if (threadIdx.x == 0) partial[(size_t)s * gridDim.x + blockIdx.x] = tot;
}

// out[s * ostride] = sum_b partial[s][b]
__global__ void __launch_bounds__(kT)
k_reduce_sets(const double* __restrict__ partial, int nblk, double* __restrict__ out, int ostride) {
  const int s = blockIdx.x;
  double acc = 0.0;
  for (int i = threadIdx.x; i < nblk; i += kT) acc += partial[(size_t)s * nblk + i];
  const double t = block_sum_d(acc);
  if (threadIdx.x == 0) out[(size_t)s * ostride] = t;
}

template <class T>
__global__ void k_init_zero_states(T* work, uint64_t nstate, int B) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < B) { T one; one.x = 1; one.y = 0; work[(size_t)s * nstate] = one; }
}

// ---------------------------------------------------------------- host
struct Workspace {
  void* ptr = nullptr;
  size_t bytes = 0;
};
std::mutex g_mu;
Workspace g_ws[64];

int ensure_ws(int dev, size_t bytes, void** p) {
  Workspace& w = g_ws[dev & 63];
  if (w.bytes < bytes) {
    if (w.ptr) cudaFree(w.ptr);
    w.ptr = nullptr;
    w.bytes = 0;
    cudaError_t e = cudaMalloc(&w.ptr, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      w.ptr = nullptr;
      return e == cudaErrorMemoryAllocation ? qc_fail(QC_ERR_OOM, "adjoint workspace of %zu bytes", bytes)
                                            : qc_cuda_fail(e, "cudaMalloc(adjoint workspace)");
    }
    w.bytes = bytes;
  }
  *p = w.ptr;
  return QC_OK;
}

bool is_param(const qc_gate& g) {
  return (g.kind == QC_GATE_RX || g.kind == QC_GATE_RY || g.kind == QC_GATE_RZ) && g.nc == 0;
}

int grid_x(uint64_t work, int states) {
  const uint64_t want = (work + kT * 4 - 1) / (kT * 4);
  const uint64_t cap = std::max<uint64_t>(1, (uint64_t)qc_num_sms() * 32 / std::max(1, states));
  return (int)std::max<uint64_t>(1, std::min(want, cap));
}

int build_hterms(int n, const qc_pauli_sum* H, HTerms& h) {
  std::memset(&h, 0, sizeof(h));
  if (!H || H->nterms < 0) return qc_fail(QC_ERR_ARG, "invalid Pauli sum");
  if (H->nterms > kMaxHTerms) return qc_fail(QC_ERR_UNSUPPORTED, "more than %d Hamiltonian terms", kMaxHTerms);
  if (H->nterms > 0 && (!H->coeffs || !H->offsets)) return qc_fail(QC_ERR_ARG, "Pauli sum arrays are NULL");
  for (int t = 0; t < H->nterms; t++) {
    if (H->offsets[t + 1] < H->offsets[t]) return qc_fail(QC_ERR_ARG, "term %d: offsets decrease", t);
    if (H->offsets[t + 1] > H->offsets[t] && (!H->letters || !H->qubits))
      return qc_fail(QC_ERR_ARG, "Pauli letters/qubits are NULL");
    uint64_t F = 0, Q = 0, used = 0;
    int ny = 0;
    for (int i = H->offsets[t]; i < H->offsets[t + 1]; i++) {
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
    h.flip[t] = F;
    h.phase[t] = Q;
    h.coeff[t] = H->coeffs[t];
    h.ipow[t] = ny & 3;
  }
  h.nterms = H->nterms;
  return QC_OK;
}

void dagger(const double* U, int D, double* out) {
  for (int r = 0; r < D; r++)
    for (int c = 0; c < D; c++) {
      out[2 * (r * D + c)] = U[2 * (c * D + r)];
      out[2 * (r * D + c) + 1] = -U[2 * (c * D + r) + 1];
    }
}

template <class Ar>
int run_adjoint(int n, const qc_gate* gates, int ngates, const double* thetas, int B, const HTerms& h,
                double* energies, double* grads, int nparams, cudaStream_t stream, int dev) {
  using coef_t = typename Ar::coef_t;
  using raw_t = typename Ar::raw_t;
  const uint64_t N = 1ull << n;
  // ---- resolve every gate (per parameter set for the parametric ones)
  struct GInfo { qc_op op; bool param; int pidx; int P; size_t fwd, adj; int mstride; };
  std::vector<GInfo> info(ngates);
  std::vector<coef_t> coefs;
  int p = 0;
  for (int l = 0; l < ngates; l++) {
    GInfo& gi = info[l];
    if (int rc = qc_gate_to_op(n, gates[l], gi.op)) return qc_fail(rc, "gate %d: %s", l, qc_last_error());
    if (gi.op.k > 2) return qc_fail(QC_ERR_UNSUPPORTED, "gate %d: adjoint path supports gates on <= 2 targets", l);
    gi.param = is_param(gates[l]);
    gi.P = gates[l].kind == QC_GATE_RX ? 0 : gates[l].kind == QC_GATE_RY ? 1 : 2;
    const int D = 1 << gi.op.k;
    double tmp[32];
    if (gi.param) {
      gi.pidx = p++;
      gi.mstride = D * D;
      gi.fwd = coefs.size();
      std::vector<qc_op> per(B);
      for (int b = 0; b < B; b++) {
        qc_gate g = gates[l];
        if (thetas) g.theta = thetas[(size_t)b * nparams + gi.pidx];
        qc_gate_to_op(n, g, per[b]);
        for (int i = 0; i < D * D; i++) coefs.push_back(Ar::make_coef(per[b].U[2 * i], per[b].U[2 * i + 1]));
      }
      gi.adj = coefs.size();
      for (int b = 0; b < B; b++) {
        dagger(per[b].U, D, tmp);
        for (int i = 0; i < D * D; i++) coefs.push_back(Ar::make_coef(tmp[2 * i], tmp[2 * i + 1]));
      }
    } else {
      gi.pidx = -1;
      gi.mstride = 0;
      gi.fwd = coefs.size();
      for (int i = 0; i < D * D; i++) coefs.push_back(Ar::make_coef(gi.op.U[2 * i], gi.op.U[2 * i + 1]));
      gi.adj = coefs.size();
      dagger(gi.op.U, D, tmp);
      for (int i = 0; i < D * D; i++) coefs.push_back(Ar::make_coef(tmp[2 * i], tmp[2 * i + 1]));
    }
  }
  // ---- workspace: [2B states][coef table][partials][energies B][grads B*P]
  const int gx_pairs = grid_x(N / 2, B);
  const int gx_full = grid_x(N, B);
  const int nblk = std::max(gx_pairs, gx_full);
  const size_t st_bytes = 2ull * B * N * sizeof(raw_t);
  const size_t coef_bytes = (coefs.size() * sizeof(coef_t) + 255) & ~(size_t)255;
  const size_t part_bytes = (size_t)B * nblk * sizeof(double);
  const size_t out_bytes = (size_t)B * (1 + std::max(1, nparams)) * sizeof(double);
  void* ws = nullptr;
  if (int rc = ensure_ws(dev, st_bytes + coef_bytes + part_bytes + out_bytes, &ws)) return rc;
  char* base = (char*)ws;
  raw_t* work = (raw_t*)base;
  coef_t* dcoef = (coef_t*)(base + st_bytes);
  double* partial = (double*)(base + st_bytes + coef_bytes);
  double* dE = (double*)(base + st_bytes + coef_bytes + part_bytes);
  double* dG = dE + B;
  QC_CUDA(cudaMemcpyAsync(dcoef, coefs.data(), coefs.size() * sizeof(coef_t), cudaMemcpyHostToDevice, stream));
  QC_CUDA(cudaMemsetAsync(work, 0, st_bytes, stream));
  k_init_zero_states<raw_t><<<(B + 127) / 128, 128, 0, stream>>>(work, N, B);
  QC_LAUNCHED("k_init_zero_states");

  auto launch_gate = [&](const GInfo& gi, size_t coef_off, int nstates) -> int {
    BGeom g;
    std::memset(&g, 0, sizeof(g));
    const qc_op& op = gi.op;
    int ins[QC_MAX_INS], ni = 0;
    for (int i = 0; i < op.k; i++) ins[ni++] = op.tpos[i];
    for (int i = 0; i < op.nc; i++) { ins[ni++] = op.cpos[i]; if (op.cval[i]) g.orval |= 1ull << op.cpos[i]; }
    std::sort(ins, ins + ni);
    g.nins = ni;
    for (int i = 0; i < ni; i++) g.ins[i] = ins[i];
    for (int r = 0; r < (1 << op.k); r++) {
      uint64_t off = 0;
      for (int i = 0; i < op.k; i++) if ((r >> (op.k - 1 - i)) & 1) off += 1ull << op.tpos[i];
      g.moff[r] = off;
    }
    g.ngroups = N >> ni;
    g.nstate = N;
    g.B = B;
    g.mstride = gi.mstride;
    dim3 grid(grid_x(g.ngroups, nstates), nstates);
    if (op.k == 1) k_bgate<Ar, 1><<<grid, kT, 0, stream>>>(work, g, dcoef + coef_off);
    else k_bgate<Ar, 2><<<grid, kT, 0, stream>>>(work, g, dcoef + coef_off);
    QC_LAUNCHED("k_bgate");
    return QC_OK;
  };

  // ---- forward sweep on phi (states 0..B-1)
  for (int l = 0; l < ngates; l++)
    if (int rc = launch_gate(info[l], info[l].fwd, B)) return rc;
  // ---- lambda = H phi, energies
  {
    dim3 grid(gx_full, B);
    k_hamiltonian<raw_t><<<grid, kT, 0, stream>>>(work, N, B, h);
    k_energy<raw_t><<<grid, kT, 0, stream>>>(work, N, B, partial);
    k_reduce_sets<<<B, kT, 0, stream>>>(partial, gx_full, dE, 1);
    QC_LAUNCHED("energy");
  }
  // ---- reverse sweep
  for (int l = ngates - 1; l >= 0; l--) {
    const GInfo& gi = info[l];
    if (gi.param) {
      dim3 grid(gx_pairs, B);
      k_adj_param<Ar><<<grid, kT, 0, stream>>>(work, N, B, gi.op.tpos[0], gi.P, dcoef + gi.adj, partial);
      k_reduce_sets<<<B, kT, 0, stream>>>(partial, gx_pairs, dG + gi.pidx, nparams);
      QC_LAUNCHED("k_adj_param");
    } else {
      if (l == 0) break;   // phi/lambda are not needed before the first gate
      if (int rc = launch_gate(gi, gi.adj, 2 * B)) return rc;
    }
  }
  QC_CUDA(cudaMemcpyAsync(energies, dE, sizeof(double) * B, cudaMemcpyDeviceToHost, stream));
  if (nparams > 0)
    QC_CUDA(cudaMemcpyAsync(grads, dG, sizeof(double) * (size_t)B * nparams, cudaMemcpyDeviceToHost, stream));
  QC_CUDA(cudaStreamSynchronize(stream));
  return QC_OK;
}

}  // namespace

extern "C" int qc_count_params(const qc_gate* gates, int ngates, int* nparams) {
  if (!nparams || ngates < 0 || (ngates > 0 && !gates)) return qc_fail(QC_ERR_ARG, "invalid arguments");
  int c = 0;
  for (int i = 0; i < ngates; i++) c += is_param(gates[i]) ? 1 : 0;
  *nparams = c;
  return QC_OK;
}

extern "C" int qc_adjoint_grad(int n, const qc_gate* gates, int ngates, const double* thetas, int batch,
                               const qc_pauli_sum* H, double* energies, double* grads, const qc_grad_opts* opts) {
  if (n < 1 || n > 34) return qc_fail(QC_ERR_ARG, "n=%d out of range 1..34", n);
  if (batch < 1 || batch > 65535) return qc_fail(QC_ERR_ARG, "batch=%d out of range 1..65535", batch);
  if (!thetas && batch != 1) return qc_fail(QC_ERR_ARG, "thetas is NULL but batch=%d", batch);
  if (!energies) return qc_fail(QC_ERR_ARG, "energies is NULL");
  int nparams = 0;
  if (int rc = qc_count_params(gates, ngates, &nparams)) return rc;
  if (nparams > 0 && !grads) return qc_fail(QC_ERR_ARG, "grads is NULL");
  const int dtype = opts ? opts->dtype : QC_C128;
  const int arith = opts ? opts->arith : QC_ARITH_AUTO;
  if (dtype != QC_C64 && dtype != QC_C128) return qc_fail(QC_ERR_ARG, "unknown dtype %d", dtype);
  HTerms h;
  if (int rc = build_hterms(n, H, h)) return rc;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return qc_fail(QC_ERR_CUDA, "no CUDA device available");
  int dev = 0;
  QC_CUDA(cudaGetDevice(&dev));
  cudaStream_t stream = opts ? (cudaStream_t)opts->stream : nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  if (dtype == QC_C64) return run_adjoint<ArC64>(n, gates, ngates, thetas, batch, h, energies, grads, nparams, stream, dev);
  if (arith == QC_ARITH_NATIVE)
    return run_adjoint<ArC128>(n, gates, ngates, thetas, batch, h, energies, grads, nparams, stream, dev);
  return run_adjoint<ArC128x>(n, gates, ngates, thetas, batch, h, energies, grads, nparams, stream, dev);
}
