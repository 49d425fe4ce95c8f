// qc_gates.cu -- gate kernels and the launcher that picks one per gate.
//
// Work decomposition.  The state is viewed as 32-byte vectors of V
// amplitudes (V = 4 for complex64, 2 for complex128; one DRAM sector).  A
// target or control at bit position p >= log2(V) selects whole vectors; one
// at p < log2(V) lives inside a vector and is resolved in registers.  A
// thread's unit of work (a "tile") is the set of 2^KH vectors that the gate's
// high targets connect; the tile's first vector index is obtained from the
// loop counter by inserting zero bits at the high target and high control
// positions -- QCLAB++ Alg. 1-3's masks m_L, m_C, m_R generalised to any
// number of positions (Sec. 2.4) -- and the control values are OR-ed in, so
// amplitudes that fail a high control are never read (Sec. 2.2, Fig. 3).
//
// Kernel families
//   k_dense  -- general 1- or 2-qubit matvec (Alg. 1 / 2 / 3, Eqs. (3), (12))
//   k_perm   -- pure permutations: Pauli X / CNOT / Toffoli (Sec. 2.1, 2.2,
//               2.4: "just a swap") and SWAP (Sec. 2.3, only b and c move)
//   k_phase  -- a phase on the amplitudes selected by a bit pattern: Z, S, T,
//               P(theta), CP, CZ, multi-controlled phases (Sec. 2.1: Z only
//               updates b_j); +-1 and +-i are applied as exact bit operations
//   k_kq     -- dense k-qubit gate, k <= 5, any placement (Sec. 2.4; used for
//               fused blocks and for very small states)
#include <algorithm>
#include <cmath>
#include <cstring>

#include "qc_common.cuh"

namespace {

constexpr int kThreads = 256;

struct Geom {
  uint64_t ntiles;          // tiles to process
  uint64_t orval;           // vector-unit OR of high control values / restricted bits
  uint64_t toff0, toff1;    // vector offsets of the high targets (MSB target first)
  int nins;                 // number of inserted positions
  int ins[QC_MAX_INS];      // inserted positions, ascending, vector units
  uint32_t lowc_mask;       // in-vector (element index) bits of low controls
  uint32_t lowc_val;
};

__device__ __forceinline__ uint64_t tile_base(const Geom& g, uint64_t j) {
  uint64_t b = j;
  for (int i = 0; i < g.nins; i++) b = qc_insert_zero(b, g.ins[i]);
  return b | g.orval;
}

__host__ __device__ constexpr int popc_c(int x) { return x == 0 ? 0 : (x & 1) + popc_c(x >> 1); }

// Place the bits of x at the set positions of mask (lowest bit first).
__host__ __device__ constexpr int deposit_c(int x, int mask) {
  int r = 0, bit = 0;
  for (int p = 0; p < 8; p++)
    if ((mask >> p) & 1) { if ((x >> bit) & 1) r |= 1 << p; bit++; }
  return r;
}

template <int KH>
__device__ __forceinline__ void tile_vectors(const Geom& g, uint64_t b, uint64_t* vi) {
  vi[0] = b;
  if constexpr (KH == 1) vi[1] = b + g.toff0;
  if constexpr (KH == 2) { vi[1] = b + g.toff1; vi[2] = b + g.toff0; vi[3] = b + g.toff0 + g.toff1; }
}

// ---------------------------------------------------------------- dense
template <class Ar, int D>
struct MatD { typename Ar::coef_t m[D * D]; };

template <class Ar, int KH, int LOWT>
__global__ void __launch_bounds__(kThreads)
k_dense(vec32* __restrict__ st, const __grid_constant__ Geom g,
        const __grid_constant__ MatD<Ar, (1 << (KH + popc_c(LOWT)))> M) {
  constexpr int KL = popc_c(LOWT);
  constexpr int D = 1 << (KH + KL);
  constexpr int NV = 1 << KH;
  using val_t = typename Ar::val_t;
  const uint64_t stride = (uint64_t)gridDim.x * kThreads;
  for (uint64_t j = (uint64_t)blockIdx.x * kThreads + threadIdx.x; j < g.ntiles; j += stride) {
    uint64_t vi[NV];
    tile_vectors<KH>(g, tile_base(g, j), vi);
    vec32 raw[NV];
#pragma unroll
    for (int r = 0; r < NV; r++) raw[r] = qc_ld32(st + vi[r]);
#pragma unroll
    for (int rest = 0; rest < Ar::V; rest++) {
      if (rest & LOWT) continue;
      if ((rest & g.lowc_mask) != g.lowc_val) continue;
      val_t in[D];
#pragma unroll
      for (int r = 0; r < D; r++) in[r] = Ar::load(raw[r >> KL], rest | deposit_c(r & ((1 << KL) - 1), LOWT));
      val_t out[D];
#pragma unroll
      for (int r = 0; r < D; r++) out[r] = Ar::template dot<D>(&M.m[r * D], in);
#pragma unroll
      for (int r = 0; r < D; r++) Ar::store(raw[r >> KL], rest | deposit_c(r & ((1 << KL) - 1), LOWT), out[r]);
    }
#pragma unroll
    for (int r = 0; r < NV; r++) qc_st32(st + vi[r], raw[r]);
  }
}

// ---------------------------------------------------------------- permutation
// KIND 0: 1-qubit X (members 0 <-> 1); KIND 1: SWAP (members 1 <-> 2).
template <int E>
__device__ __forceinline__ void swap_elems(vec32& a, int ea, vec32& b, int eb) {
  constexpr int W = E / 4;
#pragma unroll
  for (int w = 0; w < W; w++) { uint32_t t = a.w[ea * W + w]; a.w[ea * W + w] = b.w[eb * W + w]; b.w[eb * W + w] = t; }
}

template <int E, int KH, int LOWT, int KIND>
__global__ void __launch_bounds__(kThreads)
k_perm(vec32* __restrict__ st, const __grid_constant__ Geom g) {
  constexpr int V = 32 / E;
  constexpr int KL = popc_c(LOWT);
  constexpr int NV = 1 << KH;
  constexpr int M0 = KIND == 0 ? 0 : 1;   // the two members that trade places
  constexpr int M1 = KIND == 0 ? 1 : 2;
  const uint64_t stride = (uint64_t)gridDim.x * kThreads;
  for (uint64_t j = (uint64_t)blockIdx.x * kThreads + threadIdx.x; j < g.ntiles; j += stride) {
    uint64_t vi[NV];
    tile_vectors<KH>(g, tile_base(g, j), vi);
    if constexpr (KL == 0) {
      // all targets select whole vectors: move the two vectors, nothing else
      const vec32 a = qc_ld32(st + vi[M0]);
      const vec32 b = qc_ld32(st + vi[M1]);
      if (g.lowc_mask == 0) {
        qc_st32(st + vi[M0], b);
        qc_st32(st + vi[M1], a);
      } else {
        vec32 x = a, y = b;
#pragma unroll
        for (int e = 0; e < V; e++)
          if ((e & g.lowc_mask) == g.lowc_val) swap_elems<E>(x, e, y, e);
        qc_st32(st + vi[M0], x);
        qc_st32(st + vi[M1], y);
      }
    } else {
      vec32 raw[NV];
#pragma unroll
      for (int r = 0; r < NV; r++) raw[r] = qc_ld32(st + vi[r]);
#pragma unroll
      for (int rest = 0; rest < V; rest++) {
        if (rest & LOWT) continue;
        if ((rest & g.lowc_mask) != g.lowc_val) continue;
        constexpr int v0 = M0 >> KL, v1 = M1 >> KL;
        const int e0 = rest | deposit_c(M0 & ((1 << KL) - 1), LOWT);
        const int e1 = rest | deposit_c(M1 & ((1 << KL) - 1), LOWT);
        swap_elems<E>(raw[v0], e0, raw[v1], e1);
      }
#pragma unroll
      for (int r = 0; r < NV; r++) qc_st32(st + vi[r], raw[r]);
    }
  }
}

// ---------------------------------------------------------------- phase
// PH 0: general complex phase, 1: -1, 2: +i, 3: -i.
template <class Ar, int PH>
__global__ void __launch_bounds__(kThreads)
k_phase(vec32* __restrict__ st, const __grid_constant__ Geom g, const typename Ar::coef_t c) {
  constexpr int V = Ar::V;
  constexpr int W = Ar::E / 4;   // words per amplitude
  constexpr int HW = W / 2;      // words per component
  const uint64_t stride = (uint64_t)gridDim.x * kThreads;
  for (uint64_t j = (uint64_t)blockIdx.x * kThreads + threadIdx.x; j < g.ntiles; j += stride) {
    const uint64_t v = tile_base(g, j);
    vec32 x = qc_ld32(st + v);
#pragma unroll
    for (int e = 0; e < V; e++) {
      if ((e & g.lowc_mask) != g.lowc_val) continue;
      if constexpr (PH == 0) {
        const typename Ar::val_t a = Ar::load(x, e);
        Ar::store(x, e, Ar::template dot<1>(&c, &a));
      } else {
        uint32_t* re = &x.w[e * W];
        uint32_t* im = &x.w[e * W + HW];
        if constexpr (PH == 1) {          // -x: flip both sign bits
          re[HW - 1] ^= 0x80000000u; im[HW - 1] ^= 0x80000000u;
        } else {
          uint32_t tr[HW], ti[HW];
#pragma unroll
          for (int w = 0; w < HW; w++) { tr[w] = re[w]; ti[w] = im[w]; }
          if constexpr (PH == 2) {        // i*(a+ib) = -b + ia
#pragma unroll
            for (int w = 0; w < HW; w++) { re[w] = ti[w]; im[w] = tr[w]; }
            re[HW - 1] ^= 0x80000000u;
          } else {                        // -i*(a+ib) = b - ia
#pragma unroll
            for (int w = 0; w < HW; w++) { re[w] = ti[w]; im[w] = tr[w]; }
            im[HW - 1] ^= 0x80000000u;
          }
        }
      }
    }
    qc_st32(st + v, x);
  }
}

// ---------------------------------------------------------------- k-qubit
// One thread per group of 2^K amplitudes; the group is staged in shared
// memory (column per thread, conflict-free), then each output row is formed
// and written.  The matrix sits in the kernel's parameter space (uniform
// reads are broadcast).
constexpr int kThreadsK = 128;

struct GeomK {
  uint64_t ngroups;
  uint64_t orval;               // element-unit OR of control values
  uint64_t moff[32];            // element offset of group member r
  int nins;
  int ins[QC_MAX_INS];          // ascending, element units
};

template <class Ar> struct Elem;
template <> struct Elem<ArC64> {
  static __device__ __forceinline__ ArC64::val_t ld(const char* p) { float2 v = *(const float2*)p; return {v.x, v.y}; }
  static __device__ __forceinline__ void st(char* p, const ArC64::val_t& x) { *(float2*)p = make_float2(x.re, x.im); }
};
template <> struct Elem<ArC128> {
  static __device__ __forceinline__ ArC128::val_t ld(const char* p) { double2 v = *(const double2*)p; return {v.x, v.y}; }
  static __device__ __forceinline__ void st(char* p, const ArC128::val_t& x) { *(double2*)p = make_double2(x.re, x.im); }
};
template <> struct Elem<ArC128x> {
  static __device__ __forceinline__ ArC128x::val_t ld(const char* p) {
    const uint4 v = *(const uint4*)p;
    return {ArC128x::split(v.x, v.y), ArC128x::split(v.z, v.w)};
  }
  static __device__ __forceinline__ void st(char* p, const ArC128x::val_t& x) {
    const double re = ArC128x::f2d(x.re.h) + ArC128x::f2d(x.re.l);
    const double im = ArC128x::f2d(x.im.h) + ArC128x::f2d(x.im.l);
    *(double2*)p = make_double2(re, im);
  }
};

template <class Ar, int K>
__global__ void __launch_bounds__(kThreadsK)
k_kq(char* __restrict__ st, const __grid_constant__ GeomK g, const __grid_constant__ MatD<Ar, (1 << K)> M) {
  constexpr int D = 1 << K;
  using val_t = typename Ar::val_t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  val_t* sx = reinterpret_cast<val_t*>(smem_raw);   // [D][kThreadsK]
  const uint64_t stride = (uint64_t)gridDim.x * kThreadsK;
  const uint64_t j0 = (uint64_t)blockIdx.x * kThreadsK + threadIdx.x;
  for (uint64_t j = j0; j < g.ngroups; j += stride) {
    uint64_t b = j;
    for (int i = 0; i < g.nins; i++) b = qc_insert_zero(b, g.ins[i]);
    b |= g.orval;
#pragma unroll
    for (int r = 0; r < D; r++) sx[r * kThreadsK + threadIdx.x] = Elem<Ar>::ld(st + (b + g.moff[r]) * Ar::E);
#pragma unroll 1
    for (int r = 0; r < D; r++) {
      val_t xin[D];
#pragma unroll
      for (int c = 0; c < D; c++) xin[c] = sx[c * kThreadsK + threadIdx.x];
      const val_t o = Ar::template dot<D>(&M.m[r * D], xin);
      Elem<Ar>::st(st + (b + g.moff[r]) * Ar::E, o);
    }
  }
}

// ---------------------------------------------------------------- fused tiles
// Dense k-qubit block (k = 3..5, fused gates) over tiles of TG consecutive
// groups.  With the TG groups taken along the lowest free bit positions, the
// tile's amplitudes are 2^kh contiguous runs of L amplitudes (every position
// below log2 L is a varying free bit or a target, or a low control); runs are
// moved between HBM and shared memory with 32-byte vector accesses, the
// matrix is applied in shared memory (inputs of a group go to registers,
// outputs overwrite them in place), and the runs are written back.
constexpr int kThreadsF = 256;

struct GeomF {
  uint64_t ntiles;            // tiles
  uint64_t orval;             // control values (all positions)
  uint64_t hoff[32];          // start offset of run h (high-target bits)
  uint32_t loff[32];          // member r: in-run offset (low targets, low controls)
  uint32_t run_of[32];        // member r: run index
  uint32_t goff[128];         // group g: in-run offset (free low positions)
  int nins;
  int ins[QC_MAX_INS];
  int tg_log;                 // log2 TG
  int lb;                     // log2 L (run length in amplitudes)
  int kh;                     // number of runs = 2^kh
};

template <class Ar, int K>
__global__ void __launch_bounds__(kThreadsF)
k_fused(vec32* __restrict__ st, const __grid_constant__ GeomF g, const __grid_constant__ MatD<Ar, (1 << K)> M) {
  constexpr int D = 1 << K;
  using raw_t = typename Ar::raw_t;
  using val_t = typename Ar::val_t;
  extern __shared__ __align__(32) unsigned char smem_f[];
  raw_t* tile = reinterpret_cast<raw_t*>(smem_f);
  const int TG = 1 << g.tg_log;
  const uint32_t L = 1u << g.lb;
  const uint32_t run_vecs = (L * Ar::E) / 32;          // 32-byte vectors per run
  const uint32_t tile_vecs = run_vecs << g.kh;
  const int tpg = kThreadsF / TG;                      // threads per group
  const int grp = threadIdx.x % TG;
  const int rsel = threadIdx.x / TG;
  for (uint64_t T = blockIdx.x; T < g.ntiles; T += gridDim.x) {
    uint64_t base = T << g.tg_log;
    for (int i = 0; i < g.nins; i++) base = qc_insert_zero(base, g.ins[i]);
    base = (base | g.orval) & ~(uint64_t)(L - 1);     // start of run 0 (amplitude index)
    const vec32* src = st + (base * Ar::E) / 32;
    // load runs
#pragma unroll 4
    for (uint32_t v = threadIdx.x; v < tile_vecs; v += kThreadsF) {
      const uint32_t h = v / run_vecs, w = v - h * run_vecs;
      reinterpret_cast<vec32*>(tile)[v] = qc_ld32(src + (g.hoff[h] * Ar::E) / 32 + w);
    }
    __syncthreads();
    val_t in[D];
#pragma unroll
    for (int r = 0; r < D; r++) in[r] = Ar::from_raw(tile[g.run_of[r] * L + g.goff[grp] + g.loff[r]]);
    __syncthreads();
    for (int r = rsel; r < D; r += tpg)
      tile[g.run_of[r] * L + g.goff[grp] + g.loff[r]] = Ar::to_raw(Ar::template dot<D>(&M.m[r * D], in));
    __syncthreads();
#pragma unroll 4
    for (uint32_t v = threadIdx.x; v < tile_vecs; v += kThreadsF) {
      const uint32_t h = v / run_vecs, w = v - h * run_vecs;
      qc_st32(const_cast<vec32*>(src) + (g.hoff[h] * Ar::E) / 32 + w, reinterpret_cast<vec32*>(tile)[v]);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- host side
inline int grid_for(uint64_t work, int threads) {
  const uint64_t want = (work + threads - 1) / threads;
  const uint64_t cap = (uint64_t)qc_num_sms() * 16;
  return (int)std::max<uint64_t>(1, std::min(want, cap));
}

bool cis(const double* u, double re, double im) { return u[0] == re && u[1] == im; }

int phase_kind(const double* z) {
  if (z[0] == -1.0 && z[1] == 0.0) return 1;
  if (z[0] == 0.0 && z[1] == 1.0) return 2;
  if (z[0] == 0.0 && z[1] == -1.0) return 3;
  return 0;
}

struct Plan {
  int L;                     // log2(V)
  Geom g;
  int KH;
  int LOWT;
};

// Build the tile geometry: targets (descending positions, MSB first) plus
// controls; `restrict_pos/val` are extra fixed bits (phase kernel).
int build_geom(const qc_state* s, int L, const int* tpos, int k, const int* cpos, const int* cval, int nc,
               Plan& P) {
  Geom& g = P.g;
  std::memset(&g, 0, sizeof(g));
  P.L = L;
  P.KH = 0;
  P.LOWT = 0;
  int ins[QC_MAX_INS], nins = 0;
  uint64_t hoffs[2] = {0, 0};
  for (int i = 0; i < k; i++) {
    if (tpos[i] >= L) {
      hoffs[P.KH++] = 1ull << (tpos[i] - L);
      ins[nins++] = tpos[i] - L;
    } else {
      P.LOWT |= 1 << tpos[i];
    }
  }
  for (int i = 0; i < nc; i++) {
    if (cpos[i] >= L) {
      ins[nins++] = cpos[i] - L;
      if (cval[i]) g.orval |= 1ull << (cpos[i] - L);
    } else {
      g.lowc_mask |= 1u << cpos[i];
      if (cval[i]) g.lowc_val |= 1u << cpos[i];
    }
  }
  std::sort(ins, ins + nins);
  g.nins = nins;
  for (int i = 0; i < nins; i++) g.ins[i] = ins[i];
  g.toff0 = hoffs[0];
  g.toff1 = hoffs[1];
  const int free_bits = s->n - L - nins;
  if (free_bits < 0) return qc_fail(QC_ERR_ARG, "gate does not fit the state");
  g.ntiles = 1ull << free_bits;
  return QC_OK;
}

template <class Ar, int KH, int LOWT>
int launch_dense_t(qc_state* s, const Plan& P, const double* U) {
  constexpr int D = 1 << (KH + popc_c(LOWT));
  MatD<Ar, D> M;
  for (int i = 0; i < D * D; i++) M.m[i] = Ar::make_coef(U[2 * i], U[2 * i + 1]);
  k_dense<Ar, KH, LOWT><<<grid_for(P.g.ntiles, kThreads), kThreads, 0, s->stream>>>((vec32*)s->ptr, P.g, M);
  QC_LAUNCHED("k_dense");
  return QC_OK;
}

template <class Ar>
int launch_dense(qc_state* s, const Plan& P, const double* U) {
  const int key = P.KH * 16 + P.LOWT;
  if constexpr (Ar::V == 2) {
    switch (key) {
      case 0x10: return launch_dense_t<Ar, 1, 0>(s, P, U);
      case 0x01: return launch_dense_t<Ar, 0, 1>(s, P, U);
      case 0x20: return launch_dense_t<Ar, 2, 0>(s, P, U);
      case 0x11: return launch_dense_t<Ar, 1, 1>(s, P, U);
    }
  } else {
    switch (key) {
      case 0x10: return launch_dense_t<Ar, 1, 0>(s, P, U);
      case 0x01: return launch_dense_t<Ar, 0, 1>(s, P, U);
      case 0x02: return launch_dense_t<Ar, 0, 2>(s, P, U);
      case 0x20: return launch_dense_t<Ar, 2, 0>(s, P, U);
      case 0x11: return launch_dense_t<Ar, 1, 1>(s, P, U);
      case 0x12: return launch_dense_t<Ar, 1, 2>(s, P, U);
      case 0x03: return launch_dense_t<Ar, 0, 3>(s, P, U);
    }
  }
  return qc_fail(QC_ERR_ARG, "internal: no dense kernel for KH=%d LOWT=%d", P.KH, P.LOWT);
}

template <int E, int KIND>
int launch_perm(qc_state* s, const Plan& P) {
  const int key = P.KH * 16 + P.LOWT;
  const int grid = grid_for(P.g.ntiles, kThreads);
  vec32* st = (vec32*)s->ptr;
#define QC_PERM(KH_, LOWT_)                                                            \
  case (KH_ * 16 + LOWT_):                                                             \
    k_perm<E, KH_, LOWT_, KIND><<<grid, kThreads, 0, s->stream>>>(st, P.g);            \
    QC_LAUNCHED("k_perm");                                                             \
    return QC_OK;
  if constexpr (KIND == 0) {
    switch (key) { QC_PERM(1, 0) QC_PERM(0, 1) QC_PERM(0, 2) }
  } else {
    if constexpr (E == 16) {
      switch (key) { QC_PERM(2, 0) QC_PERM(1, 1) }
    } else {
      switch (key) { QC_PERM(2, 0) QC_PERM(1, 1) QC_PERM(1, 2) QC_PERM(0, 3) }
    }
  }
#undef QC_PERM
  return qc_fail(QC_ERR_ARG, "internal: no permutation kernel for KH=%d LOWT=%d", P.KH, P.LOWT);
}

template <class Ar>
int launch_phase(qc_state* s, const Plan& P, const double* z) {
  const int grid = grid_for(P.g.ntiles, kThreads);
  const typename Ar::coef_t c = Ar::make_coef(z[0], z[1]);
  vec32* st = (vec32*)s->ptr;
  switch (phase_kind(z)) {
    case 1: k_phase<Ar, 1><<<grid, kThreads, 0, s->stream>>>(st, P.g, c); break;
    case 2: k_phase<Ar, 2><<<grid, kThreads, 0, s->stream>>>(st, P.g, c); break;
    case 3: k_phase<Ar, 3><<<grid, kThreads, 0, s->stream>>>(st, P.g, c); break;
    default: k_phase<Ar, 0><<<grid, kThreads, 0, s->stream>>>(st, P.g, c); break;
  }
  QC_LAUNCHED("k_phase");
  return QC_OK;
}

template <class Ar, int K>
int launch_kq_t(qc_state* s, const qc_op& op) {
  constexpr int D = 1 << K;
  GeomK g;
  std::memset(&g, 0, sizeof(g));
  int ins[QC_MAX_INS], nins = 0;
  for (int i = 0; i < K; i++) ins[nins++] = op.tpos[i];
  for (int i = 0; i < op.nc; i++) {
    ins[nins++] = op.cpos[i];
    if (op.cval[i]) g.orval |= 1ull << op.cpos[i];
  }
  std::sort(ins, ins + nins);
  g.nins = nins;
  for (int i = 0; i < nins; i++) g.ins[i] = ins[i];
  for (int r = 0; r < D; r++) {
    uint64_t off = 0;
    for (int i = 0; i < K; i++)
      if ((r >> (K - 1 - i)) & 1) off += 1ull << op.tpos[i];
    g.moff[r] = off;
  }
  g.ngroups = 1ull << (s->n - nins);
  MatD<Ar, D> M;
  for (int i = 0; i < D * D; i++) M.m[i] = Ar::make_coef(op.U[2 * i], op.U[2 * i + 1]);
  const size_t smem = (size_t)D * kThreadsK * sizeof(typename Ar::val_t);
  static bool attr_set = false;   // per instantiation
  if (!attr_set) {
    QC_CUDA(cudaFuncSetAttribute(k_kq<Ar, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr_set = true;
  }
  k_kq<Ar, K><<<grid_for(g.ngroups, kThreadsK), kThreadsK, smem, s->stream>>>((char*)s->ptr, g, M);
  QC_LAUNCHED("k_kq");
  return QC_OK;
}

template <class Ar>
int launch_kq(qc_state* s, const qc_op& op) {
  switch (op.k) {
    case 1: return launch_kq_t<Ar, 1>(s, op);
    case 2: return launch_kq_t<Ar, 2>(s, op);
    case 3: return launch_kq_t<Ar, 3>(s, op);
    case 4: return launch_kq_t<Ar, 4>(s, op);
    case 5: return launch_kq_t<Ar, 5>(s, op);
  }
  return qc_fail(QC_ERR_ARG, "k-qubit gate with k=%d (1..5 supported)", op.k);
}


// Tile geometry for k_fused; returns false when the op does not suit it
// (fewer than 32 groups, or a tile above the shared-memory budget).
bool fused_geom(const qc_state* s, const qc_op& op, int E, GeomF& g, size_t& smem) {
  std::memset(&g, 0, sizeof(g));
  const int n = s->n, k = op.k, D = 1 << k;
  int ins[QC_MAX_INS], nins = 0;
  uint64_t used = 0;
  for (int i = 0; i < k; i++) { ins[nins++] = op.tpos[i]; used |= 1ull << op.tpos[i]; }
  for (int i = 0; i < op.nc; i++) {
    ins[nins++] = op.cpos[i];
    used |= 1ull << op.cpos[i];
    if (op.cval[i]) g.orval |= 1ull << op.cpos[i];
  }
  std::sort(ins, ins + nins);
  const int free_bits = n - nins;
  for (int tg_log = 7; tg_log >= 5; tg_log--) {
    if (tg_log > free_bits) continue;
    // the tg_log lowest free positions
    int got = 0, top = -1;
    for (int p = 0; p < n && got < tg_log; p++)
      if (!((used >> p) & 1)) { got++; top = p; }
    const int lb = top + 1;
    int kh = 0;
    for (int i = 0; i < k; i++) if (op.tpos[i] >= lb) kh++;
    const size_t bytes = ((size_t)1 << lb) * E << kh;
    if (((size_t)1 << lb) * E < 32 || bytes > 96 * 1024) continue;
    g.tg_log = tg_log;
    g.lb = lb;
    g.kh = kh;
    g.nins = nins;
    for (int i = 0; i < nins; i++) g.ins[i] = ins[i];
    g.ntiles = 1ull << (free_bits - tg_log);
    const uint64_t lmask = (1ull << lb) - 1;
    // free low positions -> group offsets
    for (int gi = 0; gi < (1 << tg_log); gi++) {
      uint64_t x = 0;
      int bit = 0;
      for (int p = 0; p < lb; p++)
        if (!((used >> p) & 1)) { if ((gi >> bit) & 1) x |= 1ull << p; bit++; }
      g.goff[gi] = (uint32_t)x;
    }
    // members: low part and run index (high targets, in target order)
    int hi_idx[QC_MAX_TARGETS], nh = 0;
    for (int i = 0; i < k; i++) if (op.tpos[i] >= lb) hi_idx[nh++] = i;
    for (int r = 0; r < D; r++) {
      uint64_t lo = g.orval & lmask;
      uint32_t run = 0;
      for (int i = 0; i < k; i++) {
        const int bitv = (r >> (k - 1 - i)) & 1;
        if (op.tpos[i] < lb) { if (bitv) lo |= 1ull << op.tpos[i]; }
      }
      for (int h = 0; h < nh; h++) {
        const int bitv = (r >> (k - 1 - hi_idx[h])) & 1;
        run |= (uint32_t)bitv << (nh - 1 - h);
      }
      g.loff[r] = (uint32_t)lo;
      g.run_of[r] = run;
    }
    for (int h = 0; h < (1 << nh); h++) {
      uint64_t off = 0;
      for (int j = 0; j < nh; j++) if ((h >> (nh - 1 - j)) & 1) off += 1ull << op.tpos[hi_idx[j]];
      g.hoff[h] = off;
    }
    smem = bytes;
    return true;
  }
  return false;
}

template <class Ar, int K>
int launch_fused_t(qc_state* s, const qc_op& op, const GeomF& g, size_t smem) {
  constexpr int D = 1 << K;
  MatD<Ar, D> M;
  for (int i = 0; i < D * D; i++) M.m[i] = Ar::make_coef(op.U[2 * i], op.U[2 * i + 1]);
  static bool attr_set = false;
  if (!attr_set) {
    QC_CUDA(cudaFuncSetAttribute(k_fused<Ar, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024));
    attr_set = true;
  }
  const uint64_t cap = (uint64_t)qc_num_sms() * 8;
  const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(g.ntiles, cap));
  k_fused<Ar, K><<<grid, kThreadsF, smem, s->stream>>>((vec32*)s->ptr, g, M);
  QC_LAUNCHED("k_fused");
  return QC_OK;
}

template <class Ar>
int launch_fused(qc_state* s, const qc_op& op, bool* done) {
  *done = false;
  GeomF g;
  size_t smem = 0;
  if (op.k < 3 || !fused_geom(s, op, Ar::E, g, smem)) return QC_OK;
  *done = true;
  switch (op.k) {
    case 3: return launch_fused_t<Ar, 3>(s, op, g, smem);
    case 4: return launch_fused_t<Ar, 4>(s, op, g, smem);
    case 5: return launch_fused_t<Ar, 5>(s, op, g, smem);
  }
  *done = false;
  return QC_OK;
}

// Reorder a 2-qubit matrix so that its first target has the higher bit position.
void order_two_qubit(qc_op& op) {
  if (op.k != 2 || op.tpos[0] > op.tpos[1]) return;
  std::swap(op.tpos[0], op.tpos[1]);
  static const int sw[4] = {0, 2, 1, 3};
  double V[32];
  for (int r = 0; r < 4; r++)
    for (int c = 0; c < 4; c++) {
      V[2 * (r * 4 + c)] = op.U[2 * (sw[r] * 4 + sw[c])];
      V[2 * (r * 4 + c) + 1] = op.U[2 * (sw[r] * 4 + sw[c]) + 1];
    }
  std::memcpy(op.U, V, sizeof(V));
}

template <class Ar>
int dispatch(qc_state* s, qc_op op) {
  constexpr int L = Ar::V == 4 ? 2 : 1;
  const int E = Ar::E;
  // Wide gates (k >= 3) and states smaller than one 32-byte vector use k_kq.
  const bool tiny = s->n < L;
  if (op.k >= 3) {
    bool done = false;
    if (int rc = launch_fused<Ar>(s, op, &done)) return rc;
    return done ? QC_OK : launch_kq<Ar>(s, op);
  }
  order_two_qubit(op);
  const double* U = op.U;
  const int D = 1 << op.k;
  bool diag = true;
  for (int r = 0; r < D; r++)
    for (int c = 0; c < D; c++)
      if (r != c && (U[2 * (r * D + c)] != 0.0 || U[2 * (r * D + c) + 1] != 0.0)) diag = false;
  Plan P;
  if (diag) {
    int nonone = 0, which = -1;
    for (int r = 0; r < D; r++)
      if (!cis(&U[2 * (r * D + r)], 1.0, 0.0)) { nonone++; which = r; }
    if (nonone == 0) return QC_OK;  // identity
    if (nonone == 1 && !tiny) {
      // Restricted phase: the targets act as extra controls with the bit
      // pattern of the one diagonal entry that differs from 1.
      int cpos[QC_MAX_CONTROLS + 2], cval[QC_MAX_CONTROLS + 2], nc = 0;
      for (int i = 0; i < op.k; i++) { cpos[nc] = op.tpos[i]; cval[nc++] = (which >> (op.k - 1 - i)) & 1; }
      for (int i = 0; i < op.nc; i++) { cpos[nc] = op.cpos[i]; cval[nc++] = op.cval[i]; }
      if (int rc = build_geom(s, L, nullptr, 0, cpos, cval, nc, P)) return rc;
      return launch_phase<Ar>(s, P, &U[2 * (which * D + which)]);
    }
  }
  if (tiny) return launch_kq<Ar>(s, op);
  if (int rc = build_geom(s, L, op.tpos, op.k, op.cpos, op.cval, op.nc, P)) return rc;
  if (op.k == 1 && cis(&U[0], 0, 0) && cis(&U[2], 1, 0) && cis(&U[4], 1, 0) && cis(&U[6], 0, 0))
    return E == 16 ? launch_perm<16, 0>(s, P) : launch_perm<8, 0>(s, P);
  if (op.k == 2) {
    static const double SW[32] = {1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 0, 0, 0,
                                  0, 0, 1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 0};
    if (std::memcmp(U, SW, sizeof(SW)) == 0 || std::equal(U, U + 32, SW))
      return E == 16 ? launch_perm<16, 1>(s, P) : launch_perm<8, 1>(s, P);
  }
  return launch_dense<Ar>(s, P, U);
}

}  // namespace

int qc_launch_op(qc_state* s, const qc_op& op) {
  if (s->dtype == QC_C64) return dispatch<ArC64>(s, op);
  if (s->arith == QC_ARITH_NATIVE) return dispatch<ArC128>(s, op);
  return dispatch<ArC128x>(s, op);
}
