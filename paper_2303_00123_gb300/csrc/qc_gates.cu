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
#include <memory>
#include <cmath>
#include <cstring>
#include <type_traits>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

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

#ifndef QC_DENSE_MINB
#define QC_DENSE_MINB 4   // resident CTAs per SM the dense sweep is compiled for
#endif
template <class Ar, int KH, int LOWT>
__global__ void __launch_bounds__(kThreads, QC_DENSE_MINB)
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
  if constexpr (KL == 0) {
    // all targets select whole vectors: move the two vectors of each tile, nothing
    // else; two tiles per iteration (four loads in flight before any store)
    auto move = [&](const uint64_t* vi, vec32 a, vec32 b) {
      if (g.lowc_mask == 0) {
        qc_st32(st + vi[M0], b);
        qc_st32(st + vi[M1], a);
      } else {
#pragma unroll
        for (int e = 0; e < V; e++)
          if ((e & g.lowc_mask) == g.lowc_val) swap_elems<E>(a, e, b, e);
        qc_st32(st + vi[M0], a);
        qc_st32(st + vi[M1], b);
      }
    };
    for (uint64_t j = (uint64_t)blockIdx.x * kThreads + threadIdx.x; j < g.ntiles; j += 2 * stride) {
      const bool two = j + stride < g.ntiles;
      uint64_t vi[NV], wi[NV];
      tile_vectors<KH>(g, tile_base(g, j), vi);
      tile_vectors<KH>(g, tile_base(g, two ? j + stride : j), wi);
      const vec32 a0 = qc_ld32(st + vi[M0]), b0 = qc_ld32(st + vi[M1]);
      const vec32 a1 = qc_ld32(st + wi[M0]), b1 = qc_ld32(st + wi[M1]);
      move(vi, a0, b0);
      if (two) move(wi, a1, b1);
    }
  } else {
    for (uint64_t j = (uint64_t)blockIdx.x * kThreads + threadIdx.x; j < g.ntiles; j += stride) {
      uint64_t vi[NV];
      tile_vectors<KH>(g, tile_base(g, j), vi);
      {
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
}

// ---------------------------------------------------------------- phase
// PH 0: general complex phase, 1: -1, 2: +i, 3: -i.
template <class Ar, int PH>
__device__ __forceinline__ void phase_vec(vec32& x, const Geom& g, const typename Ar::coef_t& c) {
  constexpr int V = Ar::V;
  constexpr int W = Ar::E / 4;   // words per amplitude
  constexpr int HW = W / 2;      // words per component
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
}

// Two tiles per iteration (both loads issued before either is used), so that
// each thread keeps two 32-byte accesses in flight.
template <class Ar, int PH>
__global__ void __launch_bounds__(kThreads)
k_phase(vec32* __restrict__ st, const __grid_constant__ Geom g, const typename Ar::coef_t c) {
  const uint64_t stride = (uint64_t)gridDim.x * kThreads;
  for (uint64_t j = (uint64_t)blockIdx.x * kThreads + threadIdx.x; j < g.ntiles; j += 2 * stride) {
    const uint64_t v0 = tile_base(g, j);
    const bool two = j + stride < g.ntiles;
    const uint64_t v1 = two ? tile_base(g, j + stride) : v0;
    vec32 x0 = qc_ld32(st + v0);
    vec32 x1 = qc_ld32(st + v1);
    phase_vec<Ar, PH>(x0, g, c);
    qc_st32(st + v0, x0);
    if (two) {
      phase_vec<Ar, PH>(x1, g, c);
      qc_st32(st + v1, x1);
    }
  }
}

// ---------------------------------------------------------------- dense 2-qubit, fixed-binade chains
// complex128 2-qubit gate (4x4 matvec per group) with the float-float
// products summed in a fixed-binade chain instead of TwoSum steps.  For
// output row r, sigma = 1.5 * 2^E with 2^E at least twice S_r * max|x|
// (S_r = sum over the row of |Re u| + |Im u|, computed on the host; max|x| =
// the largest component among the group's four inputs, so every partial sum
// is at most S_r * max|x| <= 2^E / 2): t <- fma(u, x, t) stays in [2^E, 2^(E+1)),
// t - t' is exact (Sterbenz) and fma(u, x, t - t') is the step's rounding
// error (exact up to 2^-24 of itself).  The remainders and the hi*lo cross
// terms add up in the low word, the sum is (t - sigma) + low.  Six packed
// FP32-pair instructions per complex half-product (the TwoSum form takes
// twelve): the sweep is no longer bound by the FMA pipe.  Error: about
// 2^-42 of S_r * max|x| per output (the TwoSum form: 2^-44 of the sum of the
// |products|).
struct ChainRows { int esr[4]; };              // ceil(log2(2 S_r (1 + 2^-10))) per output row

// sigma = 1.5 * 2^E, E = biased exponent e (clamped to normal floats), as a packed pair
__device__ __forceinline__ uint64_t chain_sigma2(int e) {
  e = e < 24 ? 24 : (e > 254 ? 254 : e);
  const uint32_t sb = ((uint32_t)e << 23) | 0x00400000u;
  return (uint64_t)sb | ((uint64_t)sb << 32);
}

// sum_k cf[k] * x[k] (complex, packed pairs) in a fixed-binade chain started at sig
template <int K>
__device__ __forceinline__ ArC128p::val_t chain_dot(const ArC128p::coef_t* cf, const ArC128p::val_t* x, uint64_t sig) {
  using P = ArC128p;
  uint64_t t = sig, lo = 0ull;
#pragma unroll
  for (int k = 0; k < K; k++) {
#pragma unroll
    for (int half = 0; half < 2; half++) {
      const uint64_t uh = half ? cf[k].bh : cf[k].ah, ul = half ? cf[k].bl : cf[k].al;
      const uint64_t xh = half ? P::swp(x[k].h) : x[k].h, xl = half ? P::swp(x[k].l) : x[k].l;
      const uint64_t t1 = P::fma2(uh, xh, t);
      const uint64_t rr = P::fma2(uh, xh, P::sub2(t, t1));
      t = t1;
      lo = P::fma2(ul, xh, P::fma2(uh, xl, P::add2(lo, rr)));
    }
  }
  return {P::sub2(t, sig), lo};
}

// biased exponent of the largest component (hi parts) of K packed inputs
template <int K>
__device__ __forceinline__ int chain_exp(const ArC128p::val_t* x) {
  float mx = 0.f;
#pragma unroll
  for (int k = 0; k < K; k++)
    mx = fmaxf(mx, fmaxf(fabsf(ArC128p::lo32(x[k].h)), fabsf(ArC128p::hi32(x[k].h))));
  return (int)((__float_as_uint(mx) >> 23) & 0xFFu);
}

template <int KH, int LOWT>
__global__ void __launch_bounds__(kThreads, QC_DENSE_MINB)
k_dense2c(vec32* __restrict__ st, const __grid_constant__ Geom g, const __grid_constant__ MatD<ArC128p, 4> M,
          const __grid_constant__ ChainRows cr) {
  constexpr int KL = popc_c(LOWT);
  static_assert(KH + KL == 2, "2-qubit gates");
  constexpr int D = 4;
  constexpr int NV = 1 << KH;
  using P = ArC128p;
  using val_t = P::val_t;
  const uint64_t stride = (uint64_t)gridDim.x * kThreads;
  for (uint64_t j = (uint64_t)blockIdx.x * kThreads + threadIdx.x; j < g.ntiles; j += stride) {
    uint64_t vi[NV];
    tile_vectors<KH>(g, tile_base(g, j), vi);
    vec32 raw[NV];
#pragma unroll
    for (int r = 0; r < NV; r++) raw[r] = qc_ld32(st + vi[r]);
#pragma unroll
    for (int rest = 0; rest < P::V; rest++) {
      if (rest & LOWT) continue;
      if ((rest & g.lowc_mask) != g.lowc_val) continue;
      val_t in[D];
      float mx = 0.f;
#pragma unroll
      for (int r = 0; r < D; r++) {
        in[r] = P::load(raw[r >> KL], rest | deposit_c(r & ((1 << KL) - 1), LOWT));
        mx = fmaxf(mx, fmaxf(fabsf(P::lo32(in[r].h)), fabsf(P::hi32(in[r].h))));
      }
      const int ef = (int)((__float_as_uint(mx) >> 23) & 0xFFu);
      val_t out[D];
#pragma unroll
      for (int r = 0; r < D; r++) {
        int e = ef + 1 + cr.esr[r];
        e = e < 24 ? 24 : (e > 254 ? 254 : e);
        const uint32_t sb = ((uint32_t)e << 23) | 0x00400000u;
        const uint64_t sig = (uint64_t)sb | ((uint64_t)sb << 32);
        uint64_t t = sig, lo = 0ull;
        const P::coef_t* cf = &M.m[r * D];
#pragma unroll
        for (int k = 0; k < D; k++) {
#pragma unroll
          for (int half = 0; half < 2; half++) {
            // (ur, ur) * (xr, xi), then (-ui, ui) * (xi, xr)
            const uint64_t uh = half ? cf[k].bh : cf[k].ah, ul = half ? cf[k].bl : cf[k].al;
            const uint64_t xh = half ? P::swp(in[k].h) : in[k].h, xl = half ? P::swp(in[k].l) : in[k].l;
            const uint64_t t1 = P::fma2(uh, xh, t);
            const uint64_t rr = P::fma2(uh, xh, P::sub2(t, t1));
            t = t1;
            lo = P::fma2(ul, xh, P::fma2(uh, xl, P::add2(lo, rr)));
          }
        }
        out[r] = {P::sub2(t, sig), lo};
      }
#pragma unroll
      for (int r = 0; r < D; r++) P::store(raw[r >> KL], rest | deposit_c(r & ((1 << KL) - 1), LOWT), out[r]);
    }
#pragma unroll
    for (int r = 0; r < NV; r++) qc_st32(st + vi[r], raw[r]);
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

// ---------------------------------------------------------------- fused tiles, tensor cores
// complex64 dense k-qubit block (k = 3..5) on the 5th-generation tensor cores.
// For the 128 groups of a tile, V (128 x 2D reals: Re x_0..x_{D-1}, Im ...)
// times R^T, with R = [[Ur, -Ui], [Ui, Ur]] the real form of U, gives the
// outputs (Re, Im) of every group: one M=128, N=K=2D GEMM per tile.  TF32 keeps
// 11 significant bits, so operands are split into hi + lo TF32 parts and three
// products (hi*hi + hi*lo + lo*hi) are accumulated in FP32 in tensor memory
// (about 2^-22 relative error, the precision of the FP32 state itself).
// Operands live in shared memory in the K-major, no-swizzle layout (8-row x
// 16-byte core matrices; LBO = 128 B between core matrices along K, SBO =
// (2D/4)*128 B between 8-row groups); one thread issues the tcgen05.mma
// instructions and commits them to an mbarrier; every thread then reads its
// own row of the accumulator with tcgen05.ld and stores it.  Thread g of the
// CTA owns group g of the tile for loads, stores and its accumulator row; the
// next tile's inputs are loaded before the current tile's MMAs are awaited.
static __device__ int g_tc_timeouts = 0;   // bounded mbarrier waits that gave up

// Poll limits of the MMA completion waits.  A tile's wait gives up after
// `spin` polls (kTcSpinDefault unless the state sets another limit); the
// kernel then stops taking tiles and, before it frees its tensor memory,
// waits for the MMAs it has committed with the default limit.
constexpr int kTcSpinDefault = 1 << 24;

__device__ __forceinline__ uint32_t mbar_poll(uint32_t mbar, uint32_t phase, int limit) {
  uint32_t done = 0;
  for (int it = 0; it < limit && !done; it++)
    asm volatile("{ .reg .pred q; mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2; selp.u32 %0, 1, 0, q; }"
                 : "=r"(done) : "r"(mbar), "r"(phase) : "memory");
  return done;
}

__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version for tcgen05; base offset 0; no swizzle
  return d;
}

// byte offset of element (row, col) in a K-major no-swizzle operand with KR columns
__device__ __forceinline__ uint32_t kmaj_off(int row, int col, int KR) {
  return (row >> 3) * (KR >> 2) * 128 + (col >> 2) * 128 + (row & 7) * 16 + (col & 3) * 4;
}

template <int K>
struct MatC64 { float2 u[(1 << K) * (1 << K)]; };

// tcgen05.ld of N consecutive 32-bit columns of this warp's lane block.
template <int N>
__device__ __forceinline__ void tmem_ld(uint32_t addr, uint32_t* r) {
  if constexpr (N == 16) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(addr));
  } else if constexpr (N == 8) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(addr));
  } else {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(addr));
  }
}

constexpr int kThreadsTC = 256;   // two threads per accumulator row, each owns half of the members

// CTAs per SM the kernel is compiled for: 2 at k = 5 (96 KB of operands each), 3 below
template <int K> struct TcMinB { static constexpr int v = K == 5 ? 2 : 3; };

template <int K>
__global__ void __launch_bounds__(kThreadsTC, TcMinB<K>::v)
k_fused_tc(float2* __restrict__ st, const __grid_constant__ GeomF g, const __grid_constant__ MatC64<K> U, int spin) {
  constexpr int D = 1 << K;
  constexpr int H = D / 2;                        // members per thread
  constexpr int KR = 2 * D;                       // GEMM N = K
  constexpr uint32_t NCOL = 2 * KR < 32 ? 32 : 2 * KR;   // big + small accumulators
  constexpr uint32_t SBO = (KR / 4) * 128;
  extern __shared__ __align__(1024) unsigned char smem_tc[];
  unsigned char* sAh = smem_tc;                   // 128 x KR tf32
  unsigned char* sAl = sAh + 128 * KR * 4;
  unsigned char* sBh = sAl + 128 * KR * 4;        // KR x KR tf32 (row n = output n)
  unsigned char* sBl = sBh + KR * KR * 4;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  __shared__ uint64_t s_moff[D];                  // element offset of member r within a group
  const int t = threadIdx.x;
  const int w = t >> 5;
  const int row = t & 127;                        // group within the tile = accumulator row (lane)
  const int m0 = (t >> 7) * H;                    // first member of this thread
  const uint32_t mbar_a = (uint32_t)__cvta_generic_to_shared(&mbar);
  // B = R^T in K-major form is R row by row: B[n][k] = R[n][k], R = [[Ur, -Ui], [Ui, Ur]]
  for (int i = t; i < KR * KR; i += kThreadsTC) {
    const int n = i / KR, k = i % KR;
    const float2 u = U.u[(n % D) * D + (k % D)];
    const float v = n < D ? (k < D ? u.x : -u.y) : (k < D ? u.y : u.x);
    const uint32_t hi = tf32_rna(v);
    const uint32_t lo = tf32_rna(v - __uint_as_float(hi));
    *reinterpret_cast<uint32_t*>(sBh + kmaj_off(n, k, KR)) = hi;
    *reinterpret_cast<uint32_t*>(sBl + kmaj_off(n, k, KR)) = lo;
  }
  if (t < D) s_moff[t] = g.hoff[g.run_of[t]] + g.loff[t];
  if (t == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mbar_a) : "memory");
  if (w == 0) {
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&tmem_slot);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(dst), "r"(NCOL) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(KR >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
  const uint32_t idesc2 = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)((2 * KR) >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
  const uint32_t aH = (uint32_t)__cvta_generic_to_shared(sAh), aL = (uint32_t)__cvta_generic_to_shared(sAl);
  const uint32_t bH = (uint32_t)__cvta_generic_to_shared(sBh), bL = (uint32_t)__cvta_generic_to_shared(sBl);
  const uint64_t adH = umma_desc(aH, 128, SBO), bdH = umma_desc(bH, 128, SBO);
  const uint32_t L = 1u << g.lb;
  const uint64_t* moff = s_moff + m0;             // shared-memory table (broadcast reads)
  const uint64_t goff = g.goff[row];
  auto tile_base = [&](uint64_t T) {
    uint64_t b = T << g.tg_log;
    for (int i = 0; i < g.nins; i++) b = qc_insert_zero(b, g.ins[i]);
    return ((b | g.orval) & ~(uint64_t)(L - 1)) + goff;
  };
  float2 x[H];
  uint64_t T = blockIdx.x;
  uint64_t base = 0;
  if (T < g.ntiles) {
    base = tile_base(T);
#pragma unroll
    for (int r = 0; r < H; r++) x[r] = st[base + moff[r]];
  }
  // bounded wait for the MMAs' completion; one decision for the CTA
  uint32_t phase = 0;
  auto mma_wait = [&](int limit) {
    uint32_t done = mbar_poll(mbar_a, phase, limit);
    done = __syncthreads_and(done);   // tcgen05.ld is warp-collective
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (done) phase ^= 1u;
    else if (t == 0) atomicAdd(&g_tc_timeouts, 1);
    return done != 0;
  };
  bool ok = true;
  for (; T < g.ntiles && ok; T += gridDim.x) {
    // split this thread's members into the A operands: Re -> column m0+r, Im -> column D+m0+r
#pragma unroll
    for (int part = 0; part < 2; part++) {
#pragma unroll
      for (int c4 = 0; c4 < H; c4 += 4) {
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
          const float v = part == 0 ? x[c4 + j].x : x[c4 + j].y;
          hi[j] = tf32_rna(v);
          lo[j] = tf32_rna(v - __uint_as_float(hi[j]));
        }
        const int col = part * D + m0 + c4;
        *reinterpret_cast<uint4*>(sAh + kmaj_off(row, col, KR)) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4*>(sAl + kmaj_off(row, col, KR)) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (t == 0) {
      // columns [0, KR): hi*hi; columns [KR, 2KR): hi*lo + lo*hi.  Keeping the
      // small products in their own accumulator stops the tensor core's FP32
      // accumulation from dropping their low bits against the large sum.
      // Descriptors: the start address (>> 4) is the low 14 bits and every
      // operand lies below 2^18 bytes, so an offset is one 32-bit addition.
      // Bh and Bl are stored back to back: Ah against both is one MMA of N = 2 KR
      // (hi*hi into columns [0, KR), hi*lo into [KR, 2KR)), then Al*Bh into [KR, 2KR).
#pragma unroll
      for (int p = 0; p < 2; p++) {
        const uint32_t d = p == 0 ? tmem : tmem + (uint32_t)KR;
        const uint32_t alo = (uint32_t)adH + (p == 1 ? (uint32_t)((aL - aH) >> 4) : 0u);
        const uint32_t blo = (uint32_t)bdH;
        const uint32_t id = p == 0 ? idesc2 : idesc;
#pragma unroll
        for (int kk = 0; kk < KR / 8; kk++) {
          const uint64_t ad = (adH & 0xFFFFFFFF00000000ull) | (alo + (uint32_t)(kk * 16));
          const uint64_t bd = (bdH & 0xFFFFFFFF00000000ull) | (blo + (uint32_t)(kk * 16));
          const uint32_t acc = (p == 1 || kk > 0) ? 1u : 0u;
          asm volatile("{ .reg .pred q; setp.ne.b32 q, %4, 0; tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, q; }"
                       :: "r"(d), "l"(ad), "l"(bd), "r"(id), "r"(acc) : "memory");
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(mbar_a) : "memory");
    }
    // prefetch the next tile while the tensor cores work
    const uint64_t curbase = base;
    const uint64_t Tn = T + gridDim.x;
    if (Tn < g.ntiles) {
      base = tile_base(Tn);
#pragma unroll
      for (int r = 0; r < H; r++) x[r] = st[base + moff[r]];
    }
    ok = mma_wait(spin);
    if (ok) {
      // accumulator row: columns m0..m0+H-1 = Re, D+m0.. = Im of this thread's outputs
      const uint32_t lane = tmem + ((uint32_t)(32 * (w & 3)) << 16);
      constexpr int NC = H < 16 ? H : 16;
#pragma unroll
      for (int c = 0; c < H; c += NC) {
        uint32_t re0[NC], im0[NC], re1[NC], im1[NC];
        tmem_ld<NC>(lane + (uint32_t)(m0 + c), re0);
        tmem_ld<NC>(lane + (uint32_t)(D + m0 + c), im0);
        tmem_ld<NC>(lane + (uint32_t)(KR + m0 + c), re1);
        tmem_ld<NC>(lane + (uint32_t)(KR + D + m0 + c), im1);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < NC; j++)
          st[curbase + moff[c + j]] = make_float2(__uint_as_float(re0[j]) + __uint_as_float(re1[j]),
                                                  __uint_as_float(im0[j]) + __uint_as_float(im1[j]));
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  // a wait gave up: its MMAs may still write tensor memory; wait for them (same
  // phase, default limit) before freeing it
  if (!ok) mma_wait(kTcSpinDefault);
  __syncthreads();
  if (w == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(NCOL) : "memory");
}

// ---------------------------------------------------------------- fused tiles, tensor cores, complex128
// complex128 dense k-qubit block (k = 3..5) on the tensor cores, with exact
// integer slices (the error-free splitting idea of Ozaki et al.): the same
// GEMM as k_fused_tc (128 groups x 2D reals times R^T), but every operand
// entry is written as balanced base-2^8 digits that fp16 holds exactly.
//   State (A): each entry, aligned to the largest exponent E of its group
//   (2^E <= max|x| < 2^(E+1)), is rounded to an integer q < 2^48 in units of
//   2^(E-47) and written as q = sum_s a_s 2^(8(5-s)), a_0 in [0, 256],
//   a_1..a_5 in [-128, 127], times the entry's sign; the digits are bytes of
//   q + 0x8080808080 read by integer operations.
//   Matrix (B): r 2^(7-eu) (|r| < 2^eu) = sum_t b_t 2^(-8t), t = 0..6,
//   |b_t| <= 128 (balanced: each step removes the nearest integer).
// Products of digit matrices are summed by level d = s + t <= 6 (27 of
// them) into seven FP32 accumulators in tensor memory.  A digit product is at
// most 2^15 and K <= 64, so every level sum stays below 2^23: exact.  Levels
// 0..2 are at most 2^22 and become integers by one float addition, levels 3
// and 4 by two; D5 + D6/256 is rounded the same way.  The epilogue assembles
// sum_{d<=4} D_d 2^(8(5-d)) + round(D5 + D6/256) as a 64-bit integer,
// converts it to double once and adds the scale to the exponent field.
// Error: at most half a unit of 2^(E-47) per state entry (the rounding of q)
// and about 2^-54 of the group's largest entry from the matrix digits and the
// dropped levels d >= 7.  Entries below 2^-48 of their group's largest one
// contribute nothing; groups whose largest entry is below 2^-959 give zero.
template <int K>
struct MatC128 { double2 u[(1 << K) * (1 << K)]; };

constexpr int kTcA = 6;                           // state digits
constexpr int kTcB = 7;                           // matrix digits
constexpr int kTcLev = 7;                         // accumulator levels d = s + t <= 6

// x >> s for any s (PTX clamps shift amounts above 32: the result is 0)
__device__ __forceinline__ uint32_t shr_clamp(uint32_t x, uint32_t s) {
  uint32_t r;
  asm("shr.b32 %0, %1, %2;" : "=r"(r) : "r"(x), "r"(s));
  return r;
}

// q + 0x8080808080 as (high word, low word), q = round(m / 2^(emax5 - e)) for the
// entry with high word hi, low word lo (m its 53-bit mantissa, e its exponent
// field), emax5 = the group's largest exponent field + 5.
struct TcQ { uint32_t h, l; };
__device__ __forceinline__ TcQ tc_window(uint32_t hi, uint32_t lo, int emax5) {
  const int e = (int)((hi >> 20) & 0x7FFu);
  const uint32_t mh = (hi & 0xFFFFFu) | 0x100000u;
  const uint32_t s1 = (uint32_t)(emax5 - e - 1);  // >= 4
  const uint32_t tl = s1 < 32u ? __funnelshift_r(lo, mh, s1) : shr_clamp(mh, s1 - 32u);
  const uint32_t th = shr_clamp(mh, s1);
  // (t + 1) >> 1 rounds half up; adding 2 * 0x8080808080 before the shift adds the digit offset
  const uint64_t t = (((uint64_t)th << 32) | tl) + (1ull + 2ull * 0x8080808080ull);
  return {(uint32_t)(t >> 33), (uint32_t)(t >> 1)};
}

// fp16x2 digits from two byte lanes: (w & 0x00FF00FF) | k is +-(1024 + byte)
// per half (k carries the signs); subtracting t = +-(1024 or 1152) leaves the
// signed digit, exactly.
__device__ __forceinline__ uint32_t tc_dig2(uint32_t w, uint32_t k, uint32_t t) {
  const uint32_t v = (w & 0x00FF00FFu) | k;
  uint32_t r;
  asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(r) : "r"(v), "r"(t));
  return r;
}

// the six fp16x2 words (digit s of entries a and b) for two adjacent columns
__device__ __forceinline__ void tc_digit_words(TcQ qa, TcQ qb, uint32_t hia, uint32_t hib, uint32_t* w) {
  const uint32_t k = ((hia >> 16) & 0x8000u) | (hib & 0x80000000u) | 0x64006400u;
  const uint32_t t1 = k | 0x00800080u;            // +-1152: bytes hold digit + 128
  uint32_t v0 = __byte_perm(qa.h, qb.h, 0x6521) | k;   // a_0 = q' >> 40 (9 bits)
  asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(w[0]) : "r"(v0), "r"(k));
  w[1] = tc_dig2(__byte_perm(qa.h, qb.h, 0x4400), k, t1);
  w[2] = tc_dig2(__byte_perm(qa.l, qb.l, 0x7733), k, t1);
  w[3] = tc_dig2(__byte_perm(qa.l, qb.l, 0x6622), k, t1);
  w[4] = tc_dig2(__byte_perm(qa.l, qb.l, 0x5511), k, t1);
  w[5] = tc_dig2(__byte_perm(qa.l, qb.l, 0x4400), k, t1);
}

// Nearest integer of a float |x| <= 2^22 by one addition (the bits of
// x + 1.5 * 2^23, i.e. the integer plus 0x4B400000).
__device__ __forceinline__ uint32_t tc_int22(float x) { return (uint32_t)__float_as_int(__fadd_rn(x, 12582912.f)); }

// sum_d D_d 2^(8(5-d)) (levels 0..6 of one output; integer sums, |D_d| < 2^23)
// rounded to a multiple of 2^sh, as a double times 2^scale; 0 when flush.
// Levels 0..2 (|D| <= 2^22) convert by one addition each; levels 3, 4 and the
// tail D5 + D6/256 too when every level is at most 2^22 (SMALL: K <= 32 terms),
// else they are rounded to even integers by adding 1.5 * 2^24 and each
// remainder (-1, 0 or 1, exact) moves into the next level's float.  The total
// is a 64-bit integer; shifted right by sh (|total| <= 2^(51 + sh), chosen by
// the host from the matrix) it sits in the mantissa of 1.5 * 2^52 + total,
// so one double subtraction converts it exactly (an integer-only conversion
// measured slower: the FP64 pipe is otherwise idle here, the integer pipe is not).
template <bool SMALL>
__device__ __forceinline__ double tc_assemble(const float* D, int sh, long long rnd, int scale, bool flush) {
  constexpr uint32_t C1 = 0x4B400000u;            // bits of 1.5 * 2^23
  const uint32_t b0 = tc_int22(D[0]), b1 = tc_int22(D[1]), b2 = tc_int22(D[2]);
  int Q, R;
  if constexpr (SMALL) {
    const uint32_t b3 = tc_int22(D[3]), b4 = tc_int22(D[4]);
    const uint32_t b5 = tc_int22(__fmaf_rn(D[6], 1.f / 256.f, D[5]));
    Q = (int)((b2 - C1) * 256u + (b3 - C1));
    R = (int)((b4 - C1) * 256u + (b5 - C1));
  } else {
    constexpr float M2 = 25165824.f;              // 1.5 * 2^24; bits(r) - 0x4BC00000 is half the even integer
    const float r3 = __fadd_rn(D[3], M2);
    const float e3 = __fsub_rn(D[3], __fsub_rn(r3, M2));
    const float d4 = __fmaf_rn(e3, 256.f, D[4]);
    const float r4 = __fadd_rn(d4, M2);
    const float e4 = __fsub_rn(d4, __fsub_rn(r4, M2));
    const float r5 = __fadd_rn(__fmaf_rn(e4, 256.f, __fmaf_rn(D[6], 1.f / 256.f, D[5])), M2);
    Q = (int)((b2 - C1) * 256u + ((uint32_t)__float_as_int(r3) - 0x4BC00000u) * 2u);
    R = (int)(((uint32_t)__float_as_int(r4) - 0x4BC00000u) * 512u + ((uint32_t)__float_as_int(r5) - 0x4BC00000u) * 2u);
  }
  // |P| < 2^30, |Q|, |R| < 2^31 (unsigned arithmetic: the offsets wrap)
  const int P = (int)(b0 * 256u + b1 - C1 * 257u);
  const long long tr = ((long long)P * 4294967296ll + (long long)Q * 65536 + R + rnd) >> sh;
  if (flush || tr == 0) return 0.0;
  const double y = __longlong_as_double(tr + 0x4338000000000000ll) - 6755399441055744.0;
  return __hiloint2double(__double2hiint(y) + scale * (1 << 20), __double2loint(y));
}

// byte offset of element (row, col) in a K-major no-swizzle fp16 operand with KR columns
__device__ __forceinline__ uint32_t kmaj16_off(int row, int col, int KR) {
  return (row >> 3) * (KR >> 3) * 128 + (col >> 3) * 128 + (row & 7) * 16 + (col & 7) * 2;
}

// Threads per CTA: two per accumulator row (four per row, for twice the
// warps, measured slower).
template <int K> struct Tc128Cfg {
  static constexpr int TPR = 2;                   // threads per row (group)
  static constexpr int NT = 128 * TPR;
  static constexpr int MINB = K <= 4 ? 2 : 1;     // CTAs per SM (k <= 4: 2 x 256 TMEM columns, 2 x 62 KB;
                                                  // 3 at k = 3 spilled and measured slower)
};

template <int K>
__global__ void __launch_bounds__(Tc128Cfg<K>::NT, Tc128Cfg<K>::MINB)
k_fused_tc128(double2* __restrict__ st, const __grid_constant__ GeomF g, const __grid_constant__ MatC128<K> U,
              int eu, int sh, int spin) {
  constexpr int D = 1 << K;
  constexpr int TPR = Tc128Cfg<K>::TPR, NT = Tc128Cfg<K>::NT;
  constexpr int H = D / TPR;                      // members per thread
  constexpr int KR = 2 * D;                       // GEMM N = K
  constexpr uint32_t NCOL = kTcLev * KR <= 128 ? 128 : (kTcLev * KR <= 256 ? 256 : 512);
  constexpr uint32_t SBO = (KR / 8) * 128;
  constexpr uint32_t ASZ = 128 * KR * 2, BSZ = KR * KR * 2;   // bytes per digit slice
  static_assert(H % 4 == 0, "four columns per store at least");
  extern __shared__ __align__(1024) unsigned char smem_tc[];
  unsigned char* sA = smem_tc;                    // [digit][128 x KR] fp16
  unsigned char* sB = sA + kTcA * ASZ;            // [digit][KR x KR] fp16, row n = output n
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  __shared__ uint64_t s_moff[D];
  __shared__ int s_emax[TPR][128];
  const int t = threadIdx.x;
  const int w = t >> 5;
  const int row = t & 127;
  const int part_of = t >> 7;                     // which slice of the row's members
  const int m0 = part_of * H;
  const uint32_t mbar_a = (uint32_t)__cvta_generic_to_shared(&mbar);
  // B digits: B[n][k] = R[n][k] 2^(7 - eu), R = [[Ur, -Ui], [Ui, Ur]], |R| < 2^eu
  const double uscale = __hiloint2double((1023 + 7 - eu) << 20, 0);
  for (int i = t; i < KR * KR; i += NT) {
    const int n = i / KR, k = i % KR;
    const double2 u = U.u[(n % D) * D + (k % D)];
    double r = (n < D ? (k < D ? u.x : -u.y) : (k < D ? u.y : u.x)) * uscale;
#pragma unroll
    for (int s = 0; s < kTcB; s++) {
      const double b = rint(r);
      *reinterpret_cast<__half*>(sB + s * BSZ + kmaj16_off(n, k, KR)) = __float2half_rn((float)b);
      r = (r - b) * 256.0;
    }
  }
  if (t < D) s_moff[t] = g.hoff[g.run_of[t]] + g.loff[t];
  if (t == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mbar_a) : "memory");
  if (w == 0) {
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&tmem_slot);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(dst), "r"(NCOL) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t aS = (uint32_t)__cvta_generic_to_shared(sA), bS = (uint32_t)__cvta_generic_to_shared(sB);
  const long long rnd = sh > 0 ? 1ll << (sh - 1) : 0ll;   // rounds the total to a multiple of 2^sh
  const uint32_t L = 1u << g.lb;
  const uint64_t* moff = s_moff + m0;
  const uint64_t goff = g.goff[row];
  auto tile_base = [&](uint64_t T) {
    uint64_t b = T << g.tg_log;
    for (int i = 0; i < g.nins; i++) b = qc_insert_zero(b, g.ins[i]);
    return ((b | g.orval) & ~(uint64_t)(L - 1)) + goff;
  };
  // bounded wait for the MMAs' completion; one decision for the CTA
  uint32_t phase = 0;
  auto mma_wait = [&](int limit) {
    uint32_t done = mbar_poll(mbar_a, phase, limit);
    done = __syncthreads_and(done);   // tcgen05.ld is warp-collective
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (done) phase ^= 1u;
    else if (t == 0) atomicAdd(&g_tc_timeouts, 1);
    return done != 0;
  };
  // accumulators -> doubles of the tile at obase
  auto epilogue = [&](uint64_t obase, int scale, bool flush) {
    const uint32_t lane = tmem + ((uint32_t)(32 * (w & 3)) << 16);
    constexpr int NC = 4;
#pragma unroll
    for (int c = 0; c < H; c += NC) {
      uint32_t re[kTcLev][NC], im[kTcLev][NC];
#pragma unroll
      for (int d = 0; d < kTcLev; d++) {
        tmem_ld<NC>(lane + (uint32_t)(d * KR + m0 + c), re[d]);
        tmem_ld<NC>(lane + (uint32_t)(d * KR + D + m0 + c), im[d]);
      }
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int j = 0; j < NC; j++) {
        float Dr[kTcLev], Di[kTcLev];
#pragma unroll
        for (int d = 0; d < kTcLev; d++) { Dr[d] = __uint_as_float(re[d][j]); Di[d] = __uint_as_float(im[d][j]); }
        st[obase + moff[c + j]] = make_double2(tc_assemble<(KR <= 32)>(Dr, sh, rnd, scale, flush),
                                                 tc_assemble<(KR <= 32)>(Di, sh, rnd, scale, flush));
      }
    }
  };
  // The 27 digit-matrix products (level d = sa + sb into accumulator d) as few,
  // wide MMAs: the matrix digits are stored back to back, i.e. as one K-major
  // matrix of 7 KR rows, so state digit sa against matrix digits t0 .. t0+nt-1 is
  // one MMA with N = nt KR whose accumulator columns start at level sa + t0
  // (N <= 256: k = 5 takes 9 MMAs per K step, k = 4 and 3 take 6).  Run by all of
  // warp 0, the MMAs predicated on one elected lane.  Descriptors: the start
  // address (>> 4) is the low 14 bits and every operand lies below 2^18 bytes, so
  // an offset is one 32-bit addition to the low word.
  auto issue_mma = [&]() {
    uint32_t lead;
    asm volatile("{ .reg .pred p; elect.sync _|p, 0xffffffff; selp.u32 %0, 1, 0, p; }" : "=r"(lead));
    const uint64_t adesc0 = umma_desc(aS, 128, SBO), bdesc0 = umma_desc(bS, 128, SBO);
    const uint32_t alo = (uint32_t)adesc0, ahi = (uint32_t)(adesc0 >> 32);
    const uint32_t blo = (uint32_t)bdesc0, bhi = (uint32_t)(bdesc0 >> 32);
    constexpr int TMAX = 256 / KR;                // matrix digits per MMA
#pragma unroll
    for (int sa = 0; sa < kTcA; sa++) {
#pragma unroll
      for (int t0 = 0; t0 < kTcLev - sa; t0 += TMAX) {
        const int nt = (kTcLev - sa - t0) < TMAX ? (kTcLev - sa - t0) : TMAX;
        // kind::f16: D = F32 (bit 4), A = B = F16 (formats 0), both K-major, N = nt KR, M = 128
        const uint32_t idn = (1u << 4) | ((uint32_t)((nt * KR) >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
#pragma unroll
        for (int kk = 0; kk < KR / 16; kk++) {
          const uint64_t ad = ((uint64_t)ahi << 32) | (alo + (uint32_t)((sa * ASZ + kk * 256) >> 4));
          const uint64_t bd = ((uint64_t)bhi << 32) | (blo + (uint32_t)((t0 * BSZ + kk * 256) >> 4));
          asm volatile("{ .reg .pred q, e; setp.ne.b32 q, %4, 0; setp.ne.b32 e, %5, 0;\n"
                       "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q; }"
                       :: "r"(tmem + (uint32_t)((sa + t0) * KR)), "l"(ad), "l"(bd), "r"(idn),
                          "r"((sa > 0 || kk > 0) ? 1 : 0), "r"(lead) : "memory");
        }
      }
    }
    asm volatile("{ .reg .pred e; setp.ne.b32 e, %1, 0;\n"
                 "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0]; }"
                 :: "r"(mbar_a), "r"(lead) : "memory");
  };
  // group exponent and digits of the tile held in xv; returns the output scale, sets flush
  auto make_digits = [&](const double2* xv, bool& flush) {
    int em = 0;
#pragma unroll
    for (int r = 0; r < H; r++) {
      em = max(em, (__double2hiint(xv[r].x) >> 20) & 0x7FF);
      em = max(em, (__double2hiint(xv[r].y) >> 20) & 0x7FF);
    }
    s_emax[part_of][row] = em;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < TPR; i++) em = max(em, s_emax[i][row]);
    // Re -> column m0 + r, Im -> column D + m0 + r; 16-byte stores (8 columns) where the thread has them
#pragma unroll
    for (int part = 0; part < 2; part++) {
      constexpr int CW = H >= 8 ? 8 : 4;          // columns per store
#pragma unroll
      for (int c0 = 0; c0 < H; c0 += CW) {
        uint32_t wd[CW / 2][kTcA];
#pragma unroll
        for (int j = 0; j < CW; j += 2) {
          const double va = part == 0 ? xv[c0 + j].x : xv[c0 + j].y;
          const double vb = part == 0 ? xv[c0 + j + 1].x : xv[c0 + j + 1].y;
          const uint32_t ha = (uint32_t)__double2hiint(va), hb = (uint32_t)__double2hiint(vb);
          tc_digit_words(tc_window(ha, (uint32_t)__double2loint(va), em + 5),
                         tc_window(hb, (uint32_t)__double2loint(vb), em + 5), ha, hb, wd[j / 2]);
        }
        const int col = part * D + m0 + c0;
#pragma unroll
        for (int s = 0; s < kTcA; s++) {
          if constexpr (CW == 8)
            *reinterpret_cast<uint4*>(sA + s * ASZ + kmaj16_off(row, col, KR)) =
                make_uint4(wd[0][s], wd[1][s], wd[2][s], wd[3][s]);
          else
            *reinterpret_cast<uint2*>(sA + s * ASZ + kmaj16_off(row, col, KR)) = make_uint2(wd[0][s], wd[1][s]);
        }
      }
    }
    // value = sum * 2^(E - 1077 + eu) (E: exponent field); groups below 2^-959 give zero
    flush = em + eu < 64;
    return em - 1077 + eu + sh;
  };
  // per tile: digits, MMAs (the next tile's loads in flight meanwhile), epilogue
  double2 x[H];
  uint64_t base = 0;
  if (blockIdx.x < g.ntiles) {
    base = tile_base(blockIdx.x);
#pragma unroll
    for (int r = 0; r < H; r++) x[r] = st[base + moff[r]];
  }
  bool ok = true;
  for (uint64_t T = blockIdx.x; T < g.ntiles && ok; T += gridDim.x) {
    const uint64_t cbase = base;
    bool cflush;
    const int cscale = make_digits(x, cflush);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (w == 0) issue_mma();
    const uint64_t Tn = T + gridDim.x;
    if (Tn < g.ntiles) {
      base = tile_base(Tn);
#pragma unroll
      for (int r = 0; r < H; r++) x[r] = st[base + moff[r]];
    }
    ok = mma_wait(spin);
    if (ok) epilogue(cbase, cscale, cflush);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  // a wait gave up: its MMAs may still write tensor memory; wait for them (same
  // phase, default limit) before freeing it
  if (!ok) mma_wait(kTcSpinDefault);
  __syncthreads();
  if (w == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(NCOL) : "memory");
}

// ---------------------------------------------------------------- fused tiles, complex128, warp-specialised
// The complex128 tensor-core block of k_fused_tc128 (same digits, same 27
// products, same integer epilogue, bit-identical results) as a pipeline of
// warp roles that work on different tiles at once, so that digit-making, the
// MMAs and the epilogue overlap instead of following one another:
//  * 8 producer warps, two threads per group (lanes 2g and 2g + 1 hold members
//    [0, D/2) and [D/2, D) of group g; the pair shares the group exponent by a
//    shuffle): a thread loads its members of tile i + 1 while tile i is in the
//    tensor cores and writes their digits once the A buffer is free again;
//  * 1 MMA warp: per tile and per accumulator part the digit-run MMAs of
//    k_fused_tc128 into a ring of accumulator slots.  A part is the outputs of
//    D / NP members in all 7 levels; k = 5 has two (7 x 32 columns each, two
//    slots), so the MMAs of one half overlap the epilogue of the other;
//  * 8 epilogue warps, two per tensor-memory lane quarter (each half of a
//    part's members): read a finished part, hand its slot back, assemble and
//    store the doubles.
// Hand-offs are mbarriers: A full (producers -> MMA warp), A empty (MMA commit
// -> producers), part full (MMA commit -> epilogue), part empty (epilogue ->
// MMA warp), and the rows' scales per tile (producers -> epilogue, with an
// empty barrier for reuse).  Every wait polls with a limit and is decided for
// the whole warp; a wait that reaches the limit raises the CTA's abort flag
// (counted once in g_tc_timeouts), which ends every role's loop; before the
// tensor memory is freed the MMA warp waits for the MMAs it committed.
constexpr int kTcFlushScale = -0x7fffffff - 1;   // row scale of a group whose outputs are zero

// Asynchronous 16- and 8-byte global -> shared copies (one thread's own
// staging slots; it waits for its own copies before reading them).
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"((uint32_t)__cvta_generic_to_shared(sdst)), "l"(gsrc)
               : "memory");
}
__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" :: "r"((uint32_t)__cvta_generic_to_shared(sdst)), "l"(gsrc)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

template <int K> struct Tc128WsCfg {
  static constexpr int D = 1 << K, KR = 2 * D;
  static constexpr int NP = K == 5 ? 2 : 1;           // accumulator parts per tile
  static constexpr int PM = D / NP;                   // members per part
  static constexpr int PC = 2 * PM;                   // columns per level and part (Re, Im)
  static constexpr int PCOLS = kTcLev * PC;           // tensor-memory columns per part
  static constexpr int NTS = 512 / PCOLS;             // accumulator slots (k = 5, 4: 2; k = 3: 4)
  static constexpr int NA = K == 5 ? 1 : (K == 4 ? 3 : 4);   // A buffers (96 / 48 / 24 KB each)
  static constexpr int NMS = 4;                       // row-scale slots
  static constexpr int NSTG = KR >= 32 ? 2 : 1;       // A-buffer stages (Re columns, Im columns)
  static constexpr int H = D / 2;                     // members per producer thread
  static constexpr int EM = PM / 2;                   // members per epilogue thread and part
  static constexpr int NTH = 17 * 32;                 // 8 producer + 8 epilogue warps + the MMA warp
  static constexpr uint32_t ASZ = 128u * KR * 2;      // bytes per state digit slice
  static constexpr uint32_t ASZT = kTcA * ASZ;        // bytes per A buffer
  static constexpr uint32_t BPZ = kTcB * PC * KR * 2; // bytes of matrix digits per part
  static constexpr uint32_t XSZ = 256u * H * 16;      // staging of the next tile: [member][producer] double2
  static constexpr size_t SMEM = (size_t)NA * ASZT + (size_t)NP * BPZ + XSZ;
};

// Poll an mbarrier phase for up to `limit` tries, giving up early when the
// CTA's abort flag is raised; the outcome is decided for the whole warp (all
// lanes must be present).  A wait that reaches its limit raises the flag and
// counts one time-out for the CTA.
__device__ __forceinline__ bool ws_wait(uint32_t bar, uint32_t parity, int limit, int* abort_flag) {
  uint32_t done = 0;
  for (int it = 0; it < limit && !done; it++) {
    asm volatile("{ .reg .pred q; mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2; selp.u32 %0, 1, 0, q; }"
                 : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    if (!done && (it & 31) == 31 && *(volatile int*)abort_flag) break;
  }
  done = __all_sync(0xffffffffu, done);
  if (!done && (threadIdx.x & 31) == 0) {
    if (atomicExch(abort_flag, 1) == 0) atomicAdd(&g_tc_timeouts, 1);
  }
  return done != 0;
}

__device__ __forceinline__ void ws_arrive(uint32_t bar) {
  asm volatile("{ .reg .b64 st; mbarrier.arrive.shared::cta.b64 st, [%0]; }" :: "r"(bar) : "memory");
}

__device__ __forceinline__ void ws_commit(uint32_t bar, uint32_t lead) {
  asm volatile("{ .reg .pred e; setp.ne.b32 e, %1, 0;\n"
               "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0]; }"
               :: "r"(bar), "r"(lead) : "memory");
}

template <int K>
__global__ void __launch_bounds__(Tc128WsCfg<K>::NTH, 1)
k_fused_tc128_ws(double2* __restrict__ st, const __grid_constant__ GeomF g, const __grid_constant__ MatC128<K> U,
                 int eu, int sh, int spin) {
  using C = Tc128WsCfg<K>;
  constexpr int D = C::D, KR = C::KR, NP = C::NP, PM = C::PM, PC = C::PC, H = C::H, EM = C::EM;
  constexpr int NA = C::NA, NTS = C::NTS, NMS = C::NMS;
  constexpr uint32_t SBO = (KR / 8) * 128;
  extern __shared__ __align__(1024) unsigned char smem_ws[];
  unsigned char* sA = smem_ws;                        // [buffer][digit][128 x KR] fp16
  unsigned char* sB = sA + NA * C::ASZT;              // [part][digit][PC rows x KR] fp16
  // A buffers in NSTG stages (k >= 4: the Re columns, then the Im columns of every member)
  constexpr int NSTG = C::NSTG, KPS = (KR / 16) / NSTG;   // K steps of 16 columns per stage
  __shared__ __align__(8) uint64_t bar_af[NA][NSTG], bar_ae[NA][NSTG], bar_tf[NTS], bar_te[NTS], bar_mf[NMS], bar_me[NMS];
  __shared__ __align__(8) uint64_t bar_drain;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_abort;
  __shared__ int s_scale[NMS][128];
  __shared__ uint64_t s_moff[D];
  __shared__ uint64_t s_pmoff[2][H + 1];          // producers' copy, rows apart by an odd word pair
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  auto sh_addr = [](const void* p) { return (uint32_t)__cvta_generic_to_shared(p); };
  // matrix digits: B row r of part p and digit s is output n = (r < PM ? p PM + r : D + p PM + r - PM)
  const double uscale = __hiloint2double((1023 + 7 - eu) << 20, 0);
  for (int i = t; i < KR * KR; i += C::NTH) {
    const int n = i / KR, k = i % KR;
    const double2 u = U.u[(n % D) * D + (k % D)];
    double r = (n < D ? (k < D ? u.x : -u.y) : (k < D ? u.y : u.x)) * uscale;
    const int mem = n % D, p = mem / PM, rr = (n < D ? 0 : PM) + mem % PM;
#pragma unroll
    for (int s = 0; s < kTcB; s++) {
      const double b = rint(r);
      *reinterpret_cast<__half*>(sB + kmaj16_off((p * kTcB + s) * PC + rr, k, KR)) = __float2half_rn((float)b);
      r = (r - b) * 256.0;
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (t < D) s_moff[t] = s_pmoff[t / H][t % H] = g.hoff[g.run_of[t]] + g.loff[t];
  if (t == 0) {
    s_abort = 0;
    auto init = [](uint64_t* b, uint32_t count) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"((uint32_t)__cvta_generic_to_shared(b)), "r"(count)
                   : "memory");
    };
    for (int a = 0; a < NA; a++)
      for (int z = 0; z < NSTG; z++) { init(&bar_af[a][z], 256); init(&bar_ae[a][z], 1); }
    for (int j = 0; j < NTS; j++) { init(&bar_tf[j], 1); init(&bar_te[j], 256); }
    for (int j = 0; j < NMS; j++) { init(&bar_mf[j], 256); init(&bar_me[j], 256); }
    init(&bar_drain, 1);
  }
  if (w == 16) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(sh_addr(&tmem_slot)), "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t L = 1u << g.lb;
  auto tile_base = [&](uint64_t T) {
    uint64_t b = T << g.tg_log;
    for (int i = 0; i < g.nins; i++) b = qc_insert_zero(b, g.ins[i]);
    return (b | g.orval) & ~(uint64_t)(L - 1);
  };

  if (w < 8) {
    // ------------------------------------------------ producers
    const int row = t >> 1, m0 = (t & 1) * H;
    const uint64_t goff = g.goff[row];
    // A tile's members arrive by asynchronous copies into this thread's staging
    // slots ([member][thread]: a warp's reads of one member are consecutive); the
    // next tile's copies start as soon as this tile's members are in registers, so
    // their latency overlaps the whole tile.
    double2* sX = reinterpret_cast<double2*>(sB + NP * C::BPZ);
    auto stage = [&](uint64_t Tn) {
      const uint64_t base = tile_base(Tn) + goff;
#pragma unroll
      for (int r = 0; r < H; r++) cp_async16(sX + r * 256 + t, st + base + s_pmoff[t & 1][r]);
      cp_async_commit();
    };
    double2 x[H];
    uint64_t T = blockIdx.x;
    if (T < g.ntiles) stage(T);
    for (int i = 0; T < g.ntiles; i++, T += gridDim.x) {
      cp_async_wait_all();
#pragma unroll
      for (int r = 0; r < H; r++) x[r] = sX[r * 256 + t];
      int em = 0;
#pragma unroll
      for (int r = 0; r < H; r++) {
        em = max(em, (__double2hiint(x[r].x) >> 20) & 0x7FF);
        em = max(em, (__double2hiint(x[r].y) >> 20) & 0x7FF);
      }
      // em is computed from every slot's value, so the slot reads have completed before the
      // (in-order issued) copies of the next tile may overwrite them
      asm volatile("" :: "r"(em) : "memory");
      if (T + gridDim.x < g.ntiles) stage(T + gridDim.x);
      em = max(em, __shfl_xor_sync(0xffffffffu, em, 1));
      const int a = i % NA;
      unsigned char* sAa = sA + a * C::ASZT;
      // Re -> column m0 + r, Im -> column D + m0 + r; 16-byte stores (8 columns) where the thread has them.
      // With two stages the Re columns are handed to the MMA warp before the Im columns are written.
      bool ok = true;
#pragma unroll
      for (int comp = 0; comp < 2; comp++) {
        const int z = NSTG == 2 ? comp : 0;
        if ((comp == 0 || NSTG == 2) && i >= NA &&
            !ws_wait(sh_addr(&bar_ae[a][z]), (uint32_t)((i / NA - 1) & 1), spin, &s_abort)) {
          ok = false;
          break;
        }
        constexpr int CW = H >= 8 ? 8 : 4;
#pragma unroll
        for (int c0 = 0; c0 < H; c0 += CW) {
          uint32_t wd[CW / 2][kTcA];
#pragma unroll
          for (int j = 0; j < CW; j += 2) {
            const double va = comp == 0 ? x[c0 + j].x : x[c0 + j].y;
            const double vb = comp == 0 ? x[c0 + j + 1].x : x[c0 + j + 1].y;
            const uint32_t ha = (uint32_t)__double2hiint(va), hb = (uint32_t)__double2hiint(vb);
            tc_digit_words(tc_window(ha, (uint32_t)__double2loint(va), em + 5),
                           tc_window(hb, (uint32_t)__double2loint(vb), em + 5), ha, hb, wd[j / 2]);
          }
          const int col = comp * D + m0 + c0;
#pragma unroll
          for (int s = 0; s < kTcA; s++) {
            if constexpr (CW == 8)
              *reinterpret_cast<uint4*>(sAa + s * C::ASZ + kmaj16_off(row, col, KR)) =
                  make_uint4(wd[0][s], wd[1][s], wd[2][s], wd[3][s]);
            else
              *reinterpret_cast<uint2*>(sAa + s * C::ASZ + kmaj16_off(row, col, KR)) = make_uint2(wd[0][s], wd[1][s]);
          }
        }
        if (comp == 1 || NSTG == 2) {
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          ws_arrive(sh_addr(&bar_af[a][z]));
        }
      }
      if (!ok) break;
      // the row's output scale (value = sum * 2^(E - 1077 + eu), E the exponent field; groups below 2^-959 give zero)
      const int ms = i % NMS;
      if (i >= NMS && !ws_wait(sh_addr(&bar_me[ms]), (uint32_t)((i / NMS - 1) & 1), spin, &s_abort)) break;
      if ((t & 1) == 0) s_scale[ms][row] = em + eu < 64 ? kTcFlushScale : em - 1077 + eu + sh;
      ws_arrive(sh_addr(&bar_mf[ms]));
    }
    cp_async_wait_all();
  } else if (w < 16) {
    // ------------------------------------------------ epilogue
    const int q = w & 3, ep = (w - 8) >> 2;
    const int row = 32 * q + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16);
    const uint64_t goff = g.goff[row];
    const long long rnd = sh > 0 ? 1ll << (sh - 1) : 0ll;
    bool go = true;
    uint64_t T = blockIdx.x;
    for (int i = 0; go && T < g.ntiles; i++, T += gridDim.x) {
      const int ms = i % NMS;
      if (!ws_wait(sh_addr(&bar_mf[ms]), (uint32_t)((i / NMS) & 1), spin, &s_abort)) break;
      const int sc = s_scale[ms][row];
      ws_arrive(sh_addr(&bar_me[ms]));
      const bool flush = sc == kTcFlushScale;
      const uint64_t obase = tile_base(T) + goff;
#pragma unroll 1
      for (int p = 0; p < NP; p++) {
        const int j = i * NP + p, slot = j % NTS;
        if (!ws_wait(sh_addr(&bar_tf[slot]), (uint32_t)((j / NTS) & 1), spin, &s_abort)) { go = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t pbase = lane_base + (uint32_t)(slot * C::PCOLS + ep * EM);
        constexpr int NC = 4;
#pragma unroll
        for (int c = 0; c < EM; c += NC) {
          uint32_t re[kTcLev][NC], im[kTcLev][NC];
#pragma unroll
          for (int d = 0; d < kTcLev; d++) {
            tmem_ld<NC>(pbase + (uint32_t)(d * PC + c), re[d]);
            tmem_ld<NC>(pbase + (uint32_t)(d * PC + PM + c), im[d]);
          }
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          if (c + NC >= EM) {
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            ws_arrive(sh_addr(&bar_te[slot]));
          }
#pragma unroll
          for (int jj = 0; jj < NC; jj++) {
            float Dr[kTcLev], Di[kTcLev];
#pragma unroll
            for (int d = 0; d < kTcLev; d++) { Dr[d] = __uint_as_float(re[d][jj]); Di[d] = __uint_as_float(im[d][jj]); }
            st[obase + s_moff[p * PM + ep * EM + c + jj]] =
                make_double2(tc_assemble<(KR <= 32)>(Dr, sh, rnd, sc, flush), tc_assemble<(KR <= 32)>(Di, sh, rnd, sc, flush));
          }
        }
      }
    }
  } else {
    // ------------------------------------------------ MMA warp
    uint32_t lead;
    asm volatile("{ .reg .pred p; elect.sync _|p, 0xffffffff; selp.u32 %0, 1, 0, p; }" : "=r"(lead));
    const uint32_t aS = sh_addr(sA), bS = sh_addr(sB);
    const uint64_t adesc0 = umma_desc(aS, 128, SBO), bdesc0 = umma_desc(bS, 128, SBO);
    const uint32_t alo = (uint32_t)adesc0, ahi = (uint32_t)(adesc0 >> 32);
    const uint32_t blo = (uint32_t)bdesc0, bhi = (uint32_t)(bdesc0 >> 32);
    bool go = true;
    uint64_t T = blockIdx.x;
    for (int i = 0; go && T < g.ntiles; i++, T += gridDim.x) {
      const int a = i % NA;
#pragma unroll 1
      for (int p = 0; p < NP && go; p++) {
        const int j = i * NP + p, slot = j % NTS;
        if (j >= NTS && !ws_wait(sh_addr(&bar_te[slot]), (uint32_t)((j / NTS - 1) & 1), spin, &s_abort)) {
          go = false;
          break;
        }
#pragma unroll
        for (int z = 0; z < NSTG; z++) {
          // (part 1 finds the stage's phase already complete)
          if (!ws_wait(sh_addr(&bar_af[a][z]), (uint32_t)((i / NA) & 1), spin, &s_abort)) {
            go = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          // state digit sa against matrix digits 0 .. 6 - sa: one MMA per K step, N = (7 - sa) PC,
          // accumulator columns from level sa
#pragma unroll
          for (int sa = 0; sa < kTcA; sa++) {
            const int nt = kTcLev - sa;
            const uint32_t idn = (1u << 4) | ((uint32_t)((nt * PC) >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
#pragma unroll
            for (int k2 = 0; k2 < KPS; k2++) {
              const int kk = z * KPS + k2;
              const uint64_t ad = ((uint64_t)ahi << 32) | (alo + (uint32_t)((a * C::ASZT + sa * C::ASZ + kk * 256) >> 4));
              const uint64_t bd = ((uint64_t)bhi << 32) | (blo + (uint32_t)((p * C::BPZ + kk * 256) >> 4));
              asm volatile("{ .reg .pred q, e; setp.ne.b32 q, %4, 0; setp.ne.b32 e, %5, 0;\n"
                           "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q; }"
                           :: "r"(tmem + (uint32_t)(slot * C::PCOLS + sa * PC)), "l"(ad), "l"(bd), "r"(idn),
                              "r"((sa > 0 || kk > 0) ? 1 : 0), "r"(lead) : "memory");
            }
          }
          // the last part has read this stage of the A buffer: the producers may refill it
          if (p == NP - 1) ws_commit(sh_addr(&bar_ae[a][z]), lead);
        }
        if (go) ws_commit(sh_addr(&bar_tf[slot]), lead);
      }
    }
    // every committed MMA has finished before the tensor memory is freed
    ws_commit(sh_addr(&bar_drain), lead);
    mbar_poll(sh_addr(&bar_drain), 0, kTcSpinDefault);
    __syncwarp();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (w == 16) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(512) : "memory");
  }
}

// ---------------------------------------------------------------- fused tiles, complex64, warp-specialised
// The complex64 tensor-core block of k_fused_tc (split TF32, the same three
// products into the same two accumulators, identical results) with the warp
// roles of k_fused_tc128_ws: 8 producer warps (lanes 2g, 2g + 1: the two
// halves of group g's members) load tile i + 1 and write its hi/lo operands
// into a free A buffer; the MMA warp runs the tile's MMAs into one of four
// accumulator slots (2 KR columns each); 8 epilogue warps (two per lane
// quarter) add the two accumulators of a finished slot, hand it back and
// store.  Hand-offs and bounded waits as in k_fused_tc128_ws.
template <int K> struct TcWsCfg {
  static constexpr int D = 1 << K, KR = 2 * D;
  static constexpr int ACOLS = 2 * KR;                // hi*hi and the cross products
  static constexpr int NTS = 4;                       // accumulator slots
  static constexpr uint32_t NCOL = NTS * ACOLS < 32 ? 32 : NTS * ACOLS;   // 512, 256, 128
  static constexpr int NA = K == 5 ? 2 : 4;           // A buffers (64 / 32 / 16 KB each)
  static constexpr int H = D / 2;                     // members per producer / epilogue thread
  static constexpr int NTH = 17 * 32;
  static constexpr uint32_t AHSZ = 128u * KR * 4;     // one tf32 operand (hi or lo)
  static constexpr uint32_t ASZT = 2 * AHSZ;          // bytes per A buffer
  static constexpr uint32_t BHSZ = (uint32_t)KR * KR * 4;
  static constexpr uint32_t XSZ = 256u * H * 8;       // staging of the next tile: [member][producer] float2
  static constexpr size_t SMEM = (size_t)NA * ASZT + 2 * (size_t)BHSZ + XSZ;
};

template <int K>
__global__ void __launch_bounds__(TcWsCfg<K>::NTH, 1)
k_fused_tc_ws(float2* __restrict__ st, const __grid_constant__ GeomF g, const __grid_constant__ MatC64<K> U, int spin) {
  using C = TcWsCfg<K>;
  constexpr int D = C::D, KR = C::KR, H = C::H, NA = C::NA, NTS = C::NTS;
  constexpr uint32_t SBO = (KR / 4) * 128;
  extern __shared__ __align__(1024) unsigned char smem_tw[];
  unsigned char* sA = smem_tw;                        // [buffer][hi, lo][128 x KR] tf32
  unsigned char* sBh = sA + NA * C::ASZT;             // [KR x KR] tf32 (row n = output n), then lo
  unsigned char* sBl = sBh + C::BHSZ;
  __shared__ __align__(8) uint64_t bar_af[NA], bar_ae[NA], bar_tf[NTS], bar_te[NTS];
  __shared__ __align__(8) uint64_t bar_drain;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_abort;
  __shared__ uint64_t s_moff[D];
  __shared__ uint64_t s_pmoff[2][H + 1];          // producers' copy, rows apart by an odd word pair
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  auto sh_addr = [](const void* p) { return (uint32_t)__cvta_generic_to_shared(p); };
  // B = R^T in K-major form is R row by row: B[n][k] = R[n][k], R = [[Ur, -Ui], [Ui, Ur]]
  for (int i = t; i < KR * KR; i += C::NTH) {
    const int n = i / KR, k = i % KR;
    const float2 u = U.u[(n % D) * D + (k % D)];
    const float v = n < D ? (k < D ? u.x : -u.y) : (k < D ? u.y : u.x);
    const uint32_t hi = tf32_rna(v);
    *reinterpret_cast<uint32_t*>(sBh + kmaj_off(n, k, KR)) = hi;
    *reinterpret_cast<uint32_t*>(sBl + kmaj_off(n, k, KR)) = tf32_rna(v - __uint_as_float(hi));
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (t < D) s_moff[t] = s_pmoff[t / H][t % H] = g.hoff[g.run_of[t]] + g.loff[t];
  if (t == 0) {
    s_abort = 0;
    auto init = [](uint64_t* b, uint32_t count) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"((uint32_t)__cvta_generic_to_shared(b)), "r"(count)
                   : "memory");
    };
    for (int a = 0; a < NA; a++) { init(&bar_af[a], 256); init(&bar_ae[a], 1); }
    for (int j = 0; j < NTS; j++) { init(&bar_tf[j], 1); init(&bar_te[j], 256); }
    init(&bar_drain, 1);
  }
  if (w == 16) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(sh_addr(&tmem_slot)),
                 "r"(C::NCOL) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t L = 1u << g.lb;
  auto tile_base = [&](uint64_t T) {
    uint64_t b = T << g.tg_log;
    for (int i = 0; i < g.nins; i++) b = qc_insert_zero(b, g.ins[i]);
    return (b | g.orval) & ~(uint64_t)(L - 1);
  };

  if (w < 8) {
    // ------------------------------------------------ producers
    const int row = t >> 1, m0 = (t & 1) * H;
    const uint64_t goff = g.goff[row];
    // staged tiles as in k_fused_tc128_ws ([member][thread] float2 slots)
    float2* sX = reinterpret_cast<float2*>(sBl + C::BHSZ);
    auto stage = [&](uint64_t Tn) {
      const uint64_t base = tile_base(Tn) + goff;
#pragma unroll
      for (int r = 0; r < H; r++) cp_async8(sX + r * 256 + t, st + base + s_pmoff[t & 1][r]);
      cp_async_commit();
    };
    float2 x[H];
    uint64_t T = blockIdx.x;
    if (T < g.ntiles) stage(T);
    for (int i = 0; T < g.ntiles; i++, T += gridDim.x) {
      cp_async_wait_all();
#pragma unroll
      for (int r = 0; r < H; r++) x[r] = sX[r * 256 + t];
      // a value computed from every slot's value: the slot reads have completed before the
      // (in-order issued) copies of the next tile may overwrite them
      uint32_t tok = 0;
#pragma unroll
      for (int r = 0; r < H; r++) tok |= __float_as_uint(x[r].x) ^ __float_as_uint(x[r].y);
      asm volatile("" :: "r"(tok) : "memory");
      if (T + gridDim.x < g.ntiles) stage(T + gridDim.x);
      const int a = i % NA;
      if (i >= NA && !ws_wait(sh_addr(&bar_ae[a]), (uint32_t)((i / NA - 1) & 1), spin, &s_abort)) break;
      unsigned char* sAh = sA + a * C::ASZT;
      unsigned char* sAl = sAh + C::AHSZ;
      // Re -> column m0 + r, Im -> column D + m0 + r
#pragma unroll
      for (int comp = 0; comp < 2; comp++) {
#pragma unroll
        for (int c4 = 0; c4 < H; c4 += 4) {
          uint32_t hi[4], lo[4];
#pragma unroll
          for (int j = 0; j < 4; j++) {
            const float v = comp == 0 ? x[c4 + j].x : x[c4 + j].y;
            hi[j] = tf32_rna(v);
            lo[j] = tf32_rna(v - __uint_as_float(hi[j]));
          }
          const int col = comp * D + m0 + c4;
          *reinterpret_cast<uint4*>(sAh + kmaj_off(row, col, KR)) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
          *reinterpret_cast<uint4*>(sAl + kmaj_off(row, col, KR)) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      ws_arrive(sh_addr(&bar_af[a]));
    }
    cp_async_wait_all();
  } else if (w < 16) {
    // ------------------------------------------------ epilogue: columns m = Re, D + m = Im (hi*hi), KR + ... (cross)
    const int q = w & 3, m0 = ((w - 8) >> 2) * H;
    const int row = 32 * q + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16);
    const uint64_t goff = g.goff[row];
    uint64_t T = blockIdx.x;
    for (int i = 0; T < g.ntiles; i++, T += gridDim.x) {
      const int slot = i % NTS;
      if (!ws_wait(sh_addr(&bar_tf[slot]), (uint32_t)((i / NTS) & 1), spin, &s_abort)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t obase = tile_base(T) + goff;
      const uint32_t sbase = lane_base + (uint32_t)(slot * C::ACOLS + m0);
      constexpr int NC = H < 16 ? H : 16;
#pragma unroll
      for (int c = 0; c < H; c += NC) {
        uint32_t re0[NC], im0[NC], re1[NC], im1[NC];
        tmem_ld<NC>(sbase + (uint32_t)c, re0);
        tmem_ld<NC>(sbase + (uint32_t)(D + c), im0);
        tmem_ld<NC>(sbase + (uint32_t)(KR + c), re1);
        tmem_ld<NC>(sbase + (uint32_t)(KR + D + c), im1);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (c + NC >= H) {
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          ws_arrive(sh_addr(&bar_te[slot]));
        }
#pragma unroll
        for (int j = 0; j < NC; j++)
          st[obase + s_moff[m0 + c + j]] = make_float2(__uint_as_float(re0[j]) + __uint_as_float(re1[j]),
                                                       __uint_as_float(im0[j]) + __uint_as_float(im1[j]));
      }
    }
  } else {
    // ------------------------------------------------ MMA warp: Ah x [Bh; Bl] (N = 2 KR), then Al x Bh into [KR, 2 KR)
    uint32_t lead;
    asm volatile("{ .reg .pred p; elect.sync _|p, 0xffffffff; selp.u32 %0, 1, 0, p; }" : "=r"(lead));
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(KR >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    const uint32_t idesc2 =
        (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)((2 * KR) >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    const uint64_t adesc0 = umma_desc(sh_addr(sA), 128, SBO), bdesc0 = umma_desc(sh_addr(sBh), 128, SBO);
    const uint32_t alo0 = (uint32_t)adesc0, ahi = (uint32_t)(adesc0 >> 32);
    const uint32_t blo0 = (uint32_t)bdesc0, bhi = (uint32_t)(bdesc0 >> 32);
    bool go = true;
    uint64_t T = blockIdx.x;
    for (int i = 0; go && T < g.ntiles; i++, T += gridDim.x) {
      const int a = i % NA, slot = i % NTS;
      if (!ws_wait(sh_addr(&bar_af[a]), (uint32_t)((i / NA) & 1), spin, &s_abort)) break;
      if (i >= NTS && !ws_wait(sh_addr(&bar_te[slot]), (uint32_t)((i / NTS - 1) & 1), spin, &s_abort)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int p = 0; p < 2; p++) {
        const uint32_t d = tmem + (uint32_t)(slot * C::ACOLS + (p == 0 ? 0 : KR));
        const uint32_t alo = alo0 + (uint32_t)((a * C::ASZT + (p == 1 ? C::AHSZ : 0u)) >> 4);
        const uint32_t id = p == 0 ? idesc2 : idesc;
#pragma unroll
        for (int kk = 0; kk < KR / 8; kk++) {
          const uint64_t ad = ((uint64_t)ahi << 32) | (alo + (uint32_t)(kk * 16));
          const uint64_t bd = ((uint64_t)bhi << 32) | (blo0 + (uint32_t)(kk * 16));
          asm volatile("{ .reg .pred q, e; setp.ne.b32 q, %4, 0; setp.ne.b32 e, %5, 0;\n"
                       "@e tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, q; }"
                       :: "r"(d), "l"(ad), "l"(bd), "r"(id), "r"((p == 1 || kk > 0) ? 1 : 0), "r"(lead) : "memory");
        }
      }
      ws_commit(sh_addr(&bar_tf[slot]), lead);
      ws_commit(sh_addr(&bar_ae[a]), lead);
    }
    ws_commit(sh_addr(&bar_drain), lead);
    mbar_poll(sh_addr(&bar_drain), 0, kTcSpinDefault);
    __syncwarp();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (w == 16) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(C::NCOL) : "memory");
  }
}

// ---------------------------------------------------------------- fused tiles, complex128, TMA-staged
// The complex128 tensor-core block of k_fused_tc128 with its input tiles
// staged by the Tensor Memory Accelerator.  A block without controls below
// the tile's run length has tiles of exactly 128 groups x 2^k members: 2^kh
// runs of L contiguous amplitudes.  The state is described to the TMA unit as
// a 2-D tensor of rows of 128 amplitudes (256 64-bit words), so a run is one
// box of L / 128 rows: the CTA's elected thread starts the 2^kh box loads of
// tile i + 1 (cp.async.bulk.tensor, completion counted on an mbarrier) as soon
// as every thread has read tile i out of the staging buffer, and the loads
// run while tile i's digits, MMAs and epilogue do.  No thread holds a
// prefetched tile in registers, which leaves room for TPR threads per group
// row.  Waits are bounded like the MMA waits; a CTA whose wait gave up stops
// taking tiles, waits (default limit) for its TMA loads and MMAs in flight and
// frees its tensor memory.
struct TmaGeom {
  uint32_t run_rows;          // L / 128
  uint32_t nruns;             // 2^kh
  uint32_t tile_bytes;        // 128 * 2^k * 16
};

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(mbar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1, uint32_t mbar) {
  asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
               :: "r"(dst), "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(mbar) : "memory");
}

template <int K, int TPR>
__global__ void __launch_bounds__(128 * TPR, 1)
k_fused_tc128_tma(double2* __restrict__ st, const __grid_constant__ GeomF g, const __grid_constant__ MatC128<K> U,
                  int eu, int sh, int spin, const __grid_constant__ CUtensorMap tmap, const __grid_constant__ TmaGeom tg) {
  constexpr int D = 1 << K;
  constexpr int NT = 128 * TPR;
  constexpr int H = D / TPR;                      // members per thread
  constexpr int KR = 2 * D;
  constexpr uint32_t NCOL = kTcLev * KR <= 128 ? 128 : (kTcLev * KR <= 256 ? 256 : 512);
  constexpr uint32_t SBO = (KR / 8) * 128;
  constexpr uint32_t ASZ = 128 * KR * 2, BSZ = KR * KR * 2;
  static_assert(H % 4 == 0, "four columns per store at least");
  extern __shared__ __align__(1024) unsigned char smem_tc[];
  unsigned char* sA = smem_tc;                    // [digit][128 x KR] fp16
  unsigned char* sB = sA + kTcA * ASZ;            // [digit][KR x KR] fp16
  constexpr uint32_t XOFF = ((kTcA * ASZ + kTcB * BSZ) + 1023u) & ~1023u;
  unsigned char* sX = smem_tc + XOFF;             // staging: the tile's runs back to back (16 B per amplitude)
  __shared__ __align__(8) uint64_t mbar, tbar;
  __shared__ uint32_t tmem_slot;
  __shared__ uint32_t s_moff[D];                  // member r: amplitude offset in the staging buffer
  __shared__ uint64_t s_gmoff[D];                 // member r: amplitude offset in the state from run 0's start
  __shared__ int s_emax[TPR][128];
  const int t = threadIdx.x;
  const int w = t >> 5;
  const int row = t & 127;
  const int part_of = t >> 7;
  const int m0 = part_of * H;
  const uint32_t mbar_a = (uint32_t)__cvta_generic_to_shared(&mbar);
  const uint32_t tbar_a = (uint32_t)__cvta_generic_to_shared(&tbar);
  const uint32_t sX_a = (uint32_t)__cvta_generic_to_shared(sX);
  const double uscale = __hiloint2double((1023 + 7 - eu) << 20, 0);
  for (int i = t; i < KR * KR; i += NT) {
    const int n = i / KR, k = i % KR;
    const double2 u = U.u[(n % D) * D + (k % D)];
    double r = (n < D ? (k < D ? u.x : -u.y) : (k < D ? u.y : u.x)) * uscale;
#pragma unroll
    for (int s = 0; s < kTcB; s++) {
      const double b = rint(r);
      *reinterpret_cast<__half*>(sB + s * BSZ + kmaj16_off(n, k, KR)) = __float2half_rn((float)b);
      r = (r - b) * 256.0;
    }
  }
  const uint32_t L = 1u << g.lb;
  if (t < D) {
    s_moff[t] = g.run_of[t] * L + g.loff[t];
    s_gmoff[t] = g.hoff[g.run_of[t]] + g.loff[t];
  }
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mbar_a) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(tbar_a) : "memory");
  }
  if (w == 0) {
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&tmem_slot);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(dst), "r"(NCOL) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t aS = (uint32_t)__cvta_generic_to_shared(sA), bS = (uint32_t)__cvta_generic_to_shared(sB);
  const long long rnd = sh > 0 ? 1ll << (sh - 1) : 0ll;
  const uint32_t goff = g.goff[row];
  // amplitude index of run 0 of tile T (the runs start on multiples of L >= 128)
  auto run0 = [&](uint64_t T) {
    uint64_t b = T << g.tg_log;
    for (int i = 0; i < g.nins; i++) b = qc_insert_zero(b, g.ins[i]);
    return (b | g.orval) & ~(uint64_t)(L - 1);
  };
  // elected thread: start the box loads of tile T into the staging buffer
  auto issue_tile = [&](uint64_t T) {
    const uint64_t r0 = run0(T);
    mbar_expect_tx(tbar_a, tg.tile_bytes);
    for (uint32_t h = 0; h < tg.nruns; h++)
      tma_load_2d(sX_a + h * L * 16u, &tmap, 0, (int)((r0 + g.hoff[h]) >> 7), tbar_a);
  };
  uint32_t phase = 0, tphase = 0;
  auto bar_wait = [&](uint32_t bar, uint32_t ph, int limit) {
    uint32_t done = mbar_poll(bar, ph, limit);
    done = __syncthreads_and(done);
    return done != 0;
  };
  auto mma_wait = [&](int limit) {
    const bool done = bar_wait(mbar_a, phase, limit);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (done) phase ^= 1u;
    else if (t == 0) atomicAdd(&g_tc_timeouts, 1);
    return done;
  };
  auto epilogue = [&](uint64_t obase, int scale, bool flush) {
    const uint32_t lane = tmem + ((uint32_t)(32 * (w & 3)) << 16);
    constexpr int NC = 4;
#pragma unroll
    for (int c = 0; c < H; c += NC) {
      uint32_t re[kTcLev][NC], im[kTcLev][NC];
#pragma unroll
      for (int d = 0; d < kTcLev; d++) {
        tmem_ld<NC>(lane + (uint32_t)(d * KR + m0 + c), re[d]);
        tmem_ld<NC>(lane + (uint32_t)(d * KR + D + m0 + c), im[d]);
      }
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int j = 0; j < NC; j++) {
        float Dr[kTcLev], Di[kTcLev];
#pragma unroll
        for (int d = 0; d < kTcLev; d++) { Dr[d] = __uint_as_float(re[d][j]); Di[d] = __uint_as_float(im[d][j]); }
        st[obase + s_gmoff[m0 + c + j]] = make_double2(tc_assemble<(KR <= 32)>(Dr, sh, rnd, scale, flush),
                                                         tc_assemble<(KR <= 32)>(Di, sh, rnd, scale, flush));
      }
    }
  };
  auto issue_mma = [&]() {
    uint32_t lead;
    asm volatile("{ .reg .pred p; elect.sync _|p, 0xffffffff; selp.u32 %0, 1, 0, p; }" : "=r"(lead));
    const uint64_t adesc0 = umma_desc(aS, 128, SBO), bdesc0 = umma_desc(bS, 128, SBO);
    const uint32_t alo = (uint32_t)adesc0, ahi = (uint32_t)(adesc0 >> 32);
    const uint32_t blo = (uint32_t)bdesc0, bhi = (uint32_t)(bdesc0 >> 32);
    constexpr int TMAX = 256 / KR;
#pragma unroll
    for (int sa = 0; sa < kTcA; sa++) {
#pragma unroll
      for (int t0 = 0; t0 < kTcLev - sa; t0 += TMAX) {
        const int nt = (kTcLev - sa - t0) < TMAX ? (kTcLev - sa - t0) : TMAX;
        const uint32_t idn = (1u << 4) | ((uint32_t)((nt * KR) >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
#pragma unroll
        for (int kk = 0; kk < KR / 16; kk++) {
          const uint64_t ad = ((uint64_t)ahi << 32) | (alo + (uint32_t)((sa * ASZ + kk * 256) >> 4));
          const uint64_t bd = ((uint64_t)bhi << 32) | (blo + (uint32_t)((t0 * BSZ + kk * 256) >> 4));
          asm volatile("{ .reg .pred q, e; setp.ne.b32 q, %4, 0; setp.ne.b32 e, %5, 0;\n"
                       "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q; }"
                       :: "r"(tmem + (uint32_t)((sa + t0) * KR)), "l"(ad), "l"(bd), "r"(idn),
                          "r"((sa > 0 || kk > 0) ? 1 : 0), "r"(lead) : "memory");
        }
      }
    }
    asm volatile("{ .reg .pred e; setp.ne.b32 e, %1, 0;\n"
                 "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0]; }"
                 :: "r"(mbar_a), "r"(lead) : "memory");
  };
  auto make_digits = [&](const double2* xv, bool& flush) {
    int em = 0;
#pragma unroll
    for (int r = 0; r < H; r++) {
      em = max(em, (__double2hiint(xv[r].x) >> 20) & 0x7FF);
      em = max(em, (__double2hiint(xv[r].y) >> 20) & 0x7FF);
    }
    s_emax[part_of][row] = em;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < TPR; i++) em = max(em, s_emax[i][row]);
#pragma unroll
    for (int part = 0; part < 2; part++) {
      constexpr int CW = H >= 8 ? 8 : 4;
#pragma unroll
      for (int c0 = 0; c0 < H; c0 += CW) {
        uint32_t wd[CW / 2][kTcA];
#pragma unroll
        for (int j = 0; j < CW; j += 2) {
          const double va = part == 0 ? xv[c0 + j].x : xv[c0 + j].y;
          const double vb = part == 0 ? xv[c0 + j + 1].x : xv[c0 + j + 1].y;
          const uint32_t ha = (uint32_t)__double2hiint(va), hb = (uint32_t)__double2hiint(vb);
          tc_digit_words(tc_window(ha, (uint32_t)__double2loint(va), em + 5),
                         tc_window(hb, (uint32_t)__double2loint(vb), em + 5), ha, hb, wd[j / 2]);
        }
        const int col = part * D + m0 + c0;
#pragma unroll
        for (int s = 0; s < kTcA; s++) {
          if constexpr (CW == 8)
            *reinterpret_cast<uint4*>(sA + s * ASZ + kmaj16_off(row, col, KR)) =
                make_uint4(wd[0][s], wd[1][s], wd[2][s], wd[3][s]);
          else
            *reinterpret_cast<uint2*>(sA + s * ASZ + kmaj16_off(row, col, KR)) = make_uint2(wd[0][s], wd[1][s]);
        }
      }
    }
    flush = em + eu < 64;
    return em - 1077 + eu + sh;
  };
  bool ok = true;
  bool tma_pending = false;                       // (thread 0's view) a box load is in flight
  bool mma_pending = false;                       // MMAs committed and not yet awaited
  if (t == 0 && blockIdx.x < g.ntiles) { issue_tile(blockIdx.x); tma_pending = true; }
  for (uint64_t T = blockIdx.x; T < g.ntiles && ok; T += gridDim.x) {
    // the tile's runs have landed in the staging buffer
    if (!bar_wait(tbar_a, tphase, spin)) {
      if (t == 0) atomicAdd(&g_tc_timeouts, 1);
      ok = false;
      break;
    }
    tphase ^= 1u;
    if (t == 0) tma_pending = false;
    const uint64_t cbase = run0(T) + goff;
    double2 x[H];
#pragma unroll
    for (int r = 0; r < H; r++)
      x[r] = *reinterpret_cast<const double2*>(sX + (size_t)(s_moff[m0 + r] + goff) * 16);
    bool cflush;
    const int cscale = make_digits(x, cflush);    // contains a __syncthreads: every thread has read sX
    const uint64_t Tn = T + gridDim.x;
    if (t == 0 && Tn < g.ntiles) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic reads before the async writes
      issue_tile(Tn);
      tma_pending = true;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (w == 0) issue_mma();
    mma_pending = true;
    ok = mma_wait(spin);
    if (ok) {
      mma_pending = false;
      epilogue(cbase, cscale, cflush);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  // a wait gave up: the MMAs and box loads in flight still write this CTA's memory;
  // wait for them (same phases, default limit) before freeing the tensor memory and exiting
  if (!ok) {
    if (mma_pending) mma_wait(kTcSpinDefault);
    if (__syncthreads_or(tma_pending ? 1 : 0)) bar_wait(tbar_a, tphase, kTcSpinDefault);
  }
  __syncthreads();
  if (w == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(NCOL) : "memory");
}

// ---------------------------------------------------------------- linear phase runs
// A run of commuting phase gates that all involve one qubit (the QFT's
// controlled phases after each Hadamard, Fig. 1) is one diagonal operator:
// amplitudes with the anchor bit set get exp(i (theta0 + sum_j b_j theta_j)).
// The linear bits are split into groups of at most 8; table g holds the 2^m
// partial phases of group g (host FP64, theta0 folded into table 0), so an
// amplitude needs one table entry per group and a few complex products in the
// state's arithmetic.  Only the half of the state with the anchor bit set is
// read and written.
constexpr int kLinGroups = 5;
struct LinGeom {
  Geom g;                        // vectors with the anchor bit set
  int ngroups;
  int gbits[kLinGroups];         // bits per group
  int gcontig[kLinGroups];       // 1: positions gpos[g][0], +1, ... (one shift and mask)
  int gpos[kLinGroups][8];       // bit positions (amplitude index), lowest table bit first
  int toff[kLinGroups];          // first entry of group g in the table
};

constexpr int kLinTab = 4 * 256 + 16;   // 36 linear bits: groups of 8, 8, 8, 8, 4

template <class Ar>
struct LinTab { typename Ar::coef_t t[kLinTab]; };

template <class Ar>
__global__ void __launch_bounds__(kThreads)
k_linear_phase(vec32* __restrict__ st, const __grid_constant__ LinGeom lg, const __grid_constant__ LinTab<Ar> tab,
               int ntab) {
  constexpr int V = Ar::V;
  constexpr int L = V == 4 ? 2 : 1;
  using val_t = typename Ar::val_t;
  using coef_t = typename Ar::coef_t;
  __shared__ coef_t T[kLinTab];        // lookups diverge across a warp: shared, not constant, memory
  for (int i = threadIdx.x; i < ntab; i += kThreads) T[i] = tab.t[i];
  __syncthreads();
  const uint64_t stride = (uint64_t)gridDim.x * kThreads;
  for (uint64_t j = (uint64_t)blockIdx.x * kThreads + threadIdx.x; j < lg.g.ntiles; j += stride) {
    const uint64_t v = tile_base(lg.g, j);
    vec32 x = qc_ld32(st + v);
#pragma unroll
    for (int e = 0; e < V; e++) {
      if ((e & lg.g.lowc_mask) != lg.g.lowc_val) continue;
      const uint64_t y = (v << L) | (uint64_t)e;
      val_t a = Ar::load(x, e);
      for (int g = 0; g < lg.ngroups; g++) {
        uint32_t m;
        if (lg.gcontig[g]) {
          m = (uint32_t)(y >> lg.gpos[g][0]) & ((1u << lg.gbits[g]) - 1u);
        } else {
          m = 0;
          for (int b = 0; b < lg.gbits[g]; b++) m |= (uint32_t)((y >> lg.gpos[g][b]) & 1u) << b;
        }
        a = Ar::template dot<1>(&T[lg.toff[g] + m], &a);
      }
      Ar::store(x, e, a);
    }
    qc_st32(st + v, x);
  }
}

// ---------------------------------------------------------------- dense 1q + linear phase
// One sweep for a 1-qubit gate U on the anchor followed by a run of phase
// gates that all involve the anchor (Sec. 2.2-2.4 gates, merged): every pair
// (a0, a1) of the anchor becomes U (a0, a1), then its anchor-1 member is
// multiplied by exp(i phi(y)), phi(y) = theta0 + sum_j theta_j y_{lin_j}
// (equal for both members: the linear qubits exclude the anchor).  A thread
// takes R consecutive pairs of vectors.  The factor of the linear bits above
// its window (the L in-vector bits and the log2 R bits that index the run) is
// formed once per run from tables of <= 8 bits; the window's factor comes from
// a table of V * R entries.  The high tables use the arithmetic HiAr<Ar> (the
// scalar float-float form for the packed policy, whose coefficients are three
// times larger), converted to a coefficient of Ar once per run.
template <class Ar> struct HiAr { using type = Ar; };
template <> struct HiAr<ArC128p> { using type = ArC128x; };

template <class Ar> struct PhaseCoef;
template <> struct PhaseCoef<ArC64> {
  static __device__ __forceinline__ ArC64::val_t one() { return {1.f, 0.f}; }
  static __device__ __forceinline__ ArC64::coef_t of(const ArC64::val_t& v) { return {v.re, v.im}; }
};
template <> struct PhaseCoef<ArC128> {
  static __device__ __forceinline__ ArC128::val_t one() { return {1.0, 0.0}; }
  static __device__ __forceinline__ ArC128::coef_t of(const ArC128::val_t& v) { return {v.re, v.im}; }
};
template <> struct PhaseCoef<ArC128x> {
  static __device__ __forceinline__ ArC128x::val_t one() { return {{1.f, 0.f}, {0.f, 0.f}}; }
  static __device__ __forceinline__ ArC128x::coef_t of(const ArC128x::val_t& v) {
    return {v.re.h, v.re.l, v.im.h, v.im.l};
  }
};
template <> struct PhaseCoef<ArC128p> {
  static __device__ __forceinline__ ArC128x::val_t one() { return PhaseCoef<ArC128x>::one(); }
  static __device__ __forceinline__ ArC128p::coef_t of(const ArC128x::val_t& v) {
    const float rh = v.re.h, rl = v.re.l, ih = v.im.h, il = v.im.l;
    ArC128p::coef_t c;
    c.ah = ArC128p::pk(rh, rh); c.al = ArC128p::pk(rl, rl); c.anh = ArC128p::pk(-rh, -rh);
    c.bh = ArC128p::pk(-ih, ih); c.bl = ArC128p::pk(-il, il); c.bnh = ArC128p::pk(ih, -ih);
    return c;
  }
};

constexpr int kDlGroups = 5;                 // high tables (36 linear bits, 8 per table)
constexpr int kDlHiTab = kDlGroups * 256;
constexpr int kDlR = 4;                      // vector pairs per thread and run

struct DLGeom {
  Geom g;                                    // pairs of vectors split by the anchor
  int nhg;                                   // high tables
  int hbits[kDlGroups];
  int hcontig[kDlGroups];
  int hpos[kDlGroups][8];                    // amplitude-index bit positions, lowest first
  int hoff[kDlGroups];                       // first entry of each table
};

template <class Ar>
struct DLTab {
  typename HiAr<Ar>::type::coef_t hi[kDlHiTab];
  typename Ar::coef_t w[Ar::V * kDlR];
};

// CHAIN (packed complex128 only): the two rows and the window phase sum their
// products in fixed-binade chains (see k_dense2c); esr = ceil(log2(2 S_r (1 +
// 2^-10))) of U's rows, the window phase (|w| = 1) taking row 1's plus one.
template <class Ar, int R, bool CHAIN = false>
__global__ void __launch_bounds__(kThreads, 2)
k_dense_linphase(vec32* __restrict__ st, const __grid_constant__ DLGeom dg, const __grid_constant__ MatD<Ar, 2> M,
                 const __grid_constant__ MatD<typename HiAr<Ar>::type, 2> Mh, const __grid_constant__ DLTab<Ar> tab,
                 int nhi, int esr0, int esr1) {
  constexpr int V = Ar::V;
  constexpr int L = V == 4 ? 2 : 1;
  using Hi = typename HiAr<Ar>::type;
  using val_t = typename Ar::val_t;
  __shared__ typename Hi::coef_t Th[kDlHiTab];
  __shared__ typename Ar::coef_t Tw[V * R];
  for (int i = threadIdx.x; i < nhi; i += kThreads) Th[i] = tab.hi[i];
  for (int i = threadIdx.x; i < V * R; i += kThreads) Tw[i] = tab.w[i];
  __syncthreads();
  const uint64_t nruns = dg.g.ntiles / R;
  const uint64_t stride = (uint64_t)gridDim.x * kThreads;
  for (uint64_t jr = (uint64_t)blockIdx.x * kThreads + threadIdx.x; jr < nruns; jr += stride) {
    uint64_t vi[2];
    tile_vectors<1>(dg.g, tile_base(dg.g, jr * R), vi);   // vi[0]: anchor 0, vi[1]: anchor 1
    vec32 r0[R], r1[R];
#pragma unroll
    for (int k = 0; k < R; k++) { r0[k] = qc_ld32(st + vi[0] + k); r1[k] = qc_ld32(st + vi[1] + k); }
    // factor of the linear bits above the window: the same for the whole run
    const uint64_t y = vi[1] << L;
    typename Hi::val_t h = PhaseCoef<Ar>::one();
    for (int gi = 0; gi < dg.nhg; gi++) {
      uint32_t m;
      if (dg.hcontig[gi]) {
        m = (uint32_t)(y >> dg.hpos[gi][0]) & ((1u << dg.hbits[gi]) - 1u);
      } else {
        m = 0;
        for (int b = 0; b < dg.hbits[gi]; b++) m |= (uint32_t)((y >> dg.hpos[gi][b]) & 1u) << b;
      }
      h = Hi::template dot<1>(&Th[dg.hoff[gi] + m], &h);
    }
    // U's second row times that factor: the anchor-1 output in one dot
    typename Ar::coef_t row1[2];
#pragma unroll
    for (int c = 0; c < 2; c++) row1[c] = PhaseCoef<Ar>::of(Hi::template dot<1>(&Mh.m[2 + c], &h));
#pragma unroll
    for (int k = 0; k < R; k++) {
#pragma unroll
      for (int e = 0; e < V; e++) {
        val_t in[2] = {Ar::load(r0[k], e), Ar::load(r1[k], e)};
        val_t o0, o1;
        if constexpr (CHAIN) {
          const int ef = chain_exp<2>(in);
          o0 = chain_dot<2>(&M.m[0], in, chain_sigma2(ef + 1 + esr0));
          o1 = chain_dot<2>(row1, in, chain_sigma2(ef + 1 + esr1));
          o1 = chain_dot<1>(&Tw[k * V + e], &o1, chain_sigma2(ef + 2 + esr1));
        } else {
          o0 = Ar::template dot<2>(&M.m[0], in);
          o1 = Ar::template dot<2>(row1, in);
          o1 = Ar::template dot<1>(&Tw[k * V + e], &o1);
        }
        Ar::store(r0[k], e, o0);
        Ar::store(r1[k], e, o1);
      }
    }
#pragma unroll
    for (int k = 0; k < R; k++) { qc_st32(st + vi[0] + k, r0[k]); qc_st32(st + vi[1] + k, r1[k]); }
  }
}

// ---------------------------------------------------------------- bit permutation
// A run of SWAP gates on disjoint qubit pairs (Sec. 2.3's SWAP, merged): the
// bit permutation pi swaps the paired bit positions of every basis index and
// is its own inverse.  Tile bits T = [0, t) + pi([0, t)): pi maps T onto T,
// so a tile (fixed values of the bits outside T) lands on the tile whose
// outside bits are permuted by pi; a CTA takes such a pair of tiles (or one
// tile mapped onto itself), reads both and writes both, so the update is in
// place.  Reads and writes both run over segments of 2^t contiguous
// amplitudes; the gather between them goes through shared memory, guided by
// a table src[u] = local index (in the source tile) of output local index u.
constexpr int kPermT = 5;                     // low tile bits: segments of 2^5 amplitudes
constexpr int kPermMaxTile = 1 << (2 * kPermT); // amplitudes per tile (t low bits + <= t more)
constexpr int kPermBatch = kThreads;          // tile pairs resolved per batch

struct PermGeom {
  int t, h;                                   // low bits, high tile bits
  int hpos[kPermT];                           // high tile bit positions (ascending)
  int nins;                                   // tile bit positions, ascending (for the deposit)
  int ins[2 * kPermT];
  int npairs;                                 // pairs of outside bits, as indices of the compressed tile number
  int pa[18], pb[18];
  uint64_t ntiles;
};
struct PermTab { uint16_t src[kPermMaxTile]; };

// Shared-memory slot of tile entry l: the segment number (l >> t) XORed into
// the 16-byte bank group, so that the gather, which reads entries of
// different segments at equal offsets (a transpose, for the bit reversal),
// and the segment-wise copies are both free of bank conflicts.  complex64
// keeps entry pairs (one 16-byte chunk) together.
template <int E>
__device__ __forceinline__ uint32_t perm_slot(uint32_t l, int t) {
  constexpr int S = E == 16 ? 0 : 1;
  return l ^ (((l >> t) & 7u) << S);
}

// Copies of one tile into shared memory: 16-byte cp.async chunks (a chunk
// holds 16 / E amplitudes and never straddles a 2^t segment).
template <int E>
__device__ __forceinline__ void perm_issue(const unsigned char* __restrict__ st, uint64_t f, const uint64_t* hdep,
                                           uint32_t ntile, int t, uint32_t sdst) {
  constexpr int CA = 16 / E;
  const uint32_t lowm = (1u << t) - 1u;
  for (uint32_t c = threadIdx.x; c < ntile / CA; c += kThreads) {
    const uint32_t u = c * CA;
    const uint64_t y = f | hdep[u >> t] | (u & lowm);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                 :: "r"(sdst + perm_slot<E>(u, t) * (uint32_t)E), "l"(st + y * E) : "memory");
  }
}

template <int E>
__global__ void __launch_bounds__(kThreads)
k_permute(vec32* __restrict__ st, const __grid_constant__ PermGeom pg, const __grid_constant__ PermTab tab) {
  constexpr int VA = 32 / E;                  // amplitudes per 32-byte vector
  constexpr int W = E / 4;                    // words per amplitude
  extern __shared__ __align__(16) unsigned char psm[];
  const uint32_t ntile = 1u << (pg.t + pg.h);
  // two stages, each holding a tile and its partner
  uint32_t* buf = (uint32_t*)psm;             // [stage][A|B][ntile * W]
  uint16_t* src = (uint16_t*)(buf + 4 * ntile * W);
  uint64_t* hdep = (uint64_t*)(((uintptr_t)(src + ntile) + 7) & ~(uintptr_t)7);
  uint64_t* s_in = hdep + (1 << pg.h);
  uint64_t* s_out = s_in + kPermBatch;
  int* s_list = (int*)(s_out + kPermBatch);   // canonical pairs of the batch
  int* s_cnt = s_list + kPermBatch;
  for (uint32_t i = threadIdx.x; i < ntile; i += kThreads) src[i] = tab.src[i];
  for (int c = threadIdx.x; c < (1 << pg.h); c += kThreads) {
    uint64_t d = 0;
    for (int i = 0; i < pg.h; i++) d |= (uint64_t)((c >> i) & 1) << pg.hpos[i];
    hdep[c] = d;
  }
  const unsigned char* stb = (const unsigned char*)st;
  const uint32_t sbuf = (uint32_t)__cvta_generic_to_shared(buf);
  const uint32_t tbytes = ntile * E;
  const uint32_t nvec = ntile / VA;
  const uint32_t lowm = (1u << pg.t) - 1u;
  for (uint64_t b0 = (uint64_t)blockIdx.x * kPermBatch; b0 < pg.ntiles; b0 += (uint64_t)gridDim.x * kPermBatch) {
    __syncthreads();
    {
      // tile number -> its partner, and both as fixed (outside-T) index bits
      const uint64_t tau = b0 + threadIdx.x;
      uint64_t tp = tau;
      for (int i = 0; i < pg.npairs; i++) {
        const uint64_t d = ((tp >> pg.pa[i]) ^ (tp >> pg.pb[i])) & 1ull;
        tp ^= (d << pg.pa[i]) | (d << pg.pb[i]);
      }
      uint64_t fi = tau, fo = tp;
      for (int i = 0; i < pg.nins; i++) { fi = qc_insert_zero(fi, pg.ins[i]); fo = qc_insert_zero(fo, pg.ins[i]); }
      s_in[threadIdx.x] = fi;
      s_out[threadIdx.x] = fo;
      const bool ok = tau < pg.ntiles && tau <= tp;
      // compact the canonical pairs of the batch (in tile order)
      const unsigned m = __ballot_sync(0xffffffffu, ok);
      __shared__ int wcount[kThreads / 32];
      if ((threadIdx.x & 31) == 0) wcount[threadIdx.x >> 5] = __popc(m);
      __syncthreads();
      int base = 0;
      for (int w = 0; w < (int)(threadIdx.x >> 5); w++) base += wcount[w];
      if (ok) s_list[base + __popc(m & ((1u << (threadIdx.x & 31)) - 1u))] = threadIdx.x;
      if (threadIdx.x == kThreads - 1) *s_cnt = base + __popc(m);
    }
    __syncthreads();
    const int cnt = *s_cnt;
    // pipeline: the copies of pair k + 1 are in flight while pair k is written
    if (cnt > 0) {
      const int i0 = s_list[0];
      perm_issue<E>(stb, s_in[i0], hdep, ntile, pg.t, sbuf);
      if (s_in[i0] != s_out[i0]) perm_issue<E>(stb, s_out[i0], hdep, ntile, pg.t, sbuf + tbytes);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    for (int k = 0; k < cnt; k++) {
      const int stage = k & 1;
      if (k + 1 < cnt) {
        const int i1 = s_list[k + 1];
        const uint32_t d = sbuf + (uint32_t)(stage ^ 1) * 2u * tbytes;
        perm_issue<E>(stb, s_in[i1], hdep, ntile, pg.t, d);
        if (s_in[i1] != s_out[i1]) perm_issue<E>(stb, s_out[i1], hdep, ntile, pg.t, d + tbytes);
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
      asm volatile("cp.async.wait_group 1;" ::: "memory");   // pair k's copies (this thread's)
      __syncthreads();                                        // ... and every thread's
      const int i = s_list[k];
      const uint64_t fa = s_in[i], fb = s_out[i];
      const bool two = fa != fb;
      const uint32_t* bufA = buf + (size_t)stage * 2 * ntile * W;
      const uint32_t* bufB = bufA + ntile * W;
      // A's amplitudes go to the positions of B (= pi of A's indices), and back
      for (uint32_t v = threadIdx.x; v < nvec; v += kThreads) {
        const uint32_t u = v * VA;
        const uint64_t off = hdep[u >> pg.t] | (u & lowm);
        vec32 ya, yb;
#pragma unroll
        for (int e = 0; e < VA; e++) {
          const uint32_t sidx = perm_slot<E>(src[u + e], pg.t);
          if constexpr (W == 4) {
            const uint4 a = *(const uint4*)(bufA + sidx * 4);
            ya.w[4 * e] = a.x; ya.w[4 * e + 1] = a.y; ya.w[4 * e + 2] = a.z; ya.w[4 * e + 3] = a.w;
            if (two) {
              const uint4 b = *(const uint4*)(bufB + sidx * 4);
              yb.w[4 * e] = b.x; yb.w[4 * e + 1] = b.y; yb.w[4 * e + 2] = b.z; yb.w[4 * e + 3] = b.w;
            }
          } else {
            const uint2 a = *(const uint2*)(bufA + sidx * 2);
            ya.w[2 * e] = a.x; ya.w[2 * e + 1] = a.y;
            if (two) {
              const uint2 b = *(const uint2*)(bufB + sidx * 2);
              yb.w[2 * e] = b.x; yb.w[2 * e + 1] = b.y;
            }
          }
        }
        qc_st32(st + ((fb | off) / VA), ya);
        if (two) qc_st32(st + ((fa | off) / VA), yb);
      }
      __syncthreads();                                        // stage free for pair k + 2
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
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

template <int KH, int LOWT>
int launch_dense2c_t(qc_state* s, const Plan& P, const double* U) {
  MatD<ArC128p, 4> M;
  ChainRows cr;
  for (int r = 0; r < 4; r++) {
    double S = 0.0;
    for (int c = 0; c < 4; c++) {
      M.m[r * 4 + c] = ArC128p::make_coef(U[2 * (r * 4 + c)], U[2 * (r * 4 + c) + 1]);
      S += std::fabs(U[2 * (r * 4 + c)]) + std::fabs(U[2 * (r * 4 + c) + 1]);
    }
    // 2^esr >= 2 S (a little above, so that the coefficients' and inputs' float
    // rounding is covered): every partial sum stays within 2^E / 2 of sigma
    cr.esr[r] = S > 0.0 ? (int)std::ceil(std::log2(2.0 * S * (1.0 + 0x1p-10))) : -200;
    if (S > 0.0 && (cr.esr[r] > 100 || cr.esr[r] < -100))
      return qc_fail(QC_ERR_ARG, "matrix entries out of range for the complex128 sweep");
  }
  k_dense2c<KH, LOWT><<<grid_for(P.g.ntiles, kThreads), kThreads, 0, s->stream>>>((vec32*)s->ptr, P.g, M, cr);
  QC_LAUNCHED("k_dense2c");
  return QC_OK;
}

template <class Ar>
int launch_dense(qc_state* s, const Plan& P, const double* U) {
  if constexpr (std::is_same<Ar, ArC128x>::value) {
    if (s->packed == 2) {                                    // 2-qubit gates: fixed-binade chains
      const int key2 = P.KH * 16 + P.LOWT;
      if (key2 == 0x20) return launch_dense2c_t<2, 0>(s, P, U);
      if (key2 == 0x11) return launch_dense2c_t<1, 1>(s, P, U);
    }
    if (s->packed) return launch_dense<ArC128p>(s, P, U);   // same arithmetic, packed FP32 pairs
  }
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
  if constexpr (std::is_same<Ar, ArC128x>::value) {
    if (s->packed && phase_kind(z) == 0) return launch_phase<ArC128p>(s, P, z);
  }
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
  static bool attr_set[64] = {};   // per instantiation and device (function attributes are per device)
  const int dev = s->device;
  if (dev < 0 || dev >= 64 || !attr_set[dev]) {
    QC_CUDA(cudaFuncSetAttribute(k_kq<Ar, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    QC_CUDA(cudaFuncSetAttribute(k_kq<Ar, K>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared));
    if (dev >= 0 && dev < 64) attr_set[dev] = true;
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
  static bool attr_set[64] = {};   // per device
  const int dev = s->device;
  if (dev < 0 || dev >= 64 || !attr_set[dev]) {
    QC_CUDA(cudaFuncSetAttribute(k_fused<Ar, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024));
    QC_CUDA(cudaFuncSetAttribute(k_fused<Ar, K>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared));
    if (dev >= 0 && dev < 64) attr_set[dev] = true;
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


// The state's MMA wait limit as a poll count (0 polls: every wait gives up at once).
int tc_spin(const qc_state* s) {
  if (s->wait_limit == 0) return kTcSpinDefault;
  if (s->wait_limit < 0) return 0;
  return (int)std::min<long long>(s->wait_limit, 1ll << 30);
}

template <int K>
int launch_fused_tc_ws_t(qc_state* s, const GeomF& g, const MatC64<K>& U) {
  using C = TcWsCfg<K>;
  static bool attr_set[64] = {};   // per device (function attributes are per device)
  const int sdev = s->device;
  if (sdev < 0 || sdev >= 64 || !attr_set[sdev]) {
    QC_CUDA(cudaFuncSetAttribute(k_fused_tc_ws<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM));
    QC_CUDA(cudaFuncSetAttribute(k_fused_tc_ws<K>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared));
    if (sdev >= 0 && sdev < 64) attr_set[sdev] = true;
  }
  const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(g.ntiles, (uint64_t)qc_num_sms()));
  k_fused_tc_ws<K><<<grid, C::NTH, C::SMEM, s->stream>>>((float2*)s->ptr, g, U, tc_spin(s));
  QC_LAUNCHED("k_fused_tc_ws");
  return QC_OK;
}

template <int K>
int launch_fused_tc_t(qc_state* s, const qc_op& op, const GeomF& g) {
  constexpr int D = 1 << K, KR = 2 * D;
  MatC64<K> U;
  for (int i = 0; i < D * D; i++) U.u[i] = make_float2((float)op.U[2 * i], (float)op.U[2 * i + 1]);
  // the warp-specialised pipeline only in mode 3 (the one-role kernel, two CTAs per SM, measured faster)
  if (s->fused_tc == 3) return launch_fused_tc_ws_t<K>(s, g, U);
  const size_t smem = (size_t)2 * 128 * KR * 4 + (size_t)2 * KR * KR * 4;
  static int per_sm_dev[64] = {};   // per device (function attributes are per device)
  const int sdev = s->device;
  int per_sm = sdev >= 0 && sdev < 64 ? per_sm_dev[sdev] : 0;
  if (per_sm == 0) {
    QC_CUDA(cudaFuncSetAttribute(k_fused_tc<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // the default L1/shared split caps residency at one CTA per SM; ask for the full shared memory
    QC_CUDA(cudaFuncSetAttribute(k_fused_tc<K>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared));
    // Residency from the kernel's own footprint (registers in 256-register warp
    // chunks, shared memory plus the 1 KB the runtime reserves per CTA) and the
    // tensor-memory columns each CTA allocates.
    cudaFuncAttributes fa;
    QC_CUDA(cudaFuncGetAttributes(&fa, k_fused_tc<K>));
    int dev = 0, smem_sm = 0, regs_sm = 0;
    QC_CUDA(cudaGetDevice(&dev));
    QC_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    QC_CUDA(cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev));
    const int warp_regs = ((fa.numRegs * 32 + 255) / 256) * 256;
    const int by_regs = regs_sm / (warp_regs * (kThreadsTC / 32));
    const int by_smem = smem_sm / (int)(smem + fa.sharedSizeBytes + 1024);
    const int ncol = 2 * KR < 32 ? 32 : 2 * KR;
    per_sm = std::max(1, std::min(std::min(by_regs, by_smem), std::min(512 / ncol, 2048 / kThreadsTC)));
    if (sdev >= 0 && sdev < 64) per_sm_dev[sdev] = per_sm;
  }
  const uint64_t cap = (uint64_t)qc_num_sms() * per_sm;
  const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(g.ntiles, cap));
  k_fused_tc<K><<<grid, kThreadsTC, smem, s->stream>>>((float2*)s->ptr, g, U, tc_spin(s));
  QC_LAUNCHED("k_fused_tc");
  return QC_OK;
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();
template <int K>
int launch_fused_tc128_tma_t(qc_state* s, const qc_op& op, const GeomF& g, int eu, int sh, const MatC128<K>& U);

template <int K>
int launch_fused_tc128_ws_t(qc_state* s, const GeomF& g, int eu, int sh, const MatC128<K>& U) {
  using C = Tc128WsCfg<K>;
  static bool attr_set[64] = {};   // per device (function attributes are per device)
  const int sdev = s->device;
  if (sdev < 0 || sdev >= 64 || !attr_set[sdev]) {
    QC_CUDA(cudaFuncSetAttribute(k_fused_tc128_ws<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM));
    QC_CUDA(cudaFuncSetAttribute(k_fused_tc128_ws<K>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared));
    if (sdev >= 0 && sdev < 64) attr_set[sdev] = true;
  }
  // one CTA per SM: it holds all 512 tensor-memory columns
  const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(g.ntiles, (uint64_t)qc_num_sms()));
  k_fused_tc128_ws<K><<<grid, C::NTH, C::SMEM, s->stream>>>((double2*)s->ptr, g, U, eu, sh, tc_spin(s));
  QC_LAUNCHED("k_fused_tc128_ws");
  return QC_OK;
}

template <int K>
int launch_fused_tc128_t(qc_state* s, const qc_op& op, const GeomF& g) {
  constexpr int D = 1 << K, KR = 2 * D;
  MatC128<K> U;
  double umax = 0.0;
  for (int i = 0; i < D * D; i++) {
    U.u[i] = make_double2(op.U[2 * i], op.U[2 * i + 1]);
    umax = std::max(umax, std::max(std::fabs(op.U[2 * i]), std::fabs(op.U[2 * i + 1])));
  }
  // digits of the matrix scaled by 2^(7 - eu) with |entries| < 2^eu (any matrix is allowed)
  const int eu = umax > 0.0 ? std::ilogb(umax) + 1 : 0;
  if (eu > 100 || eu < -100) return qc_fail(QC_ERR_ARG, "matrix entries out of range for the tensor-core path");
  // each output of a group, in units of its lowest level, is below S 2^(55 - eu), S the largest
  // row sum of |Re| + |Im|; the epilogue keeps it to 2^51 by dropping sh low bits
  double S = 0.0;
  for (int j = 0; j < D; j++) {
    double r = 0.0;
    for (int l = 0; l < D; l++) r += std::fabs(op.U[2 * (j * D + l)]) + std::fabs(op.U[2 * (j * D + l) + 1]);
    S = std::max(S, r);
  }
  const int sh = S > 0.0 ? std::max(0, (int)std::ceil(std::log2(S * (1.0 + 0x1p-30))) + 4 - eu) : 0;
  // TMA-staged tiles: the tile is exactly its 128 groups (no control below the run length)
  if (s->fused_tc == 2 && ((size_t)1 << g.lb << g.kh) == ((size_t)128 << K) && tensor_map_encoder())
    return launch_fused_tc128_tma_t<K>(s, op, g, eu, sh, U);
  // the warp-specialised pipeline: mode 3 always, the default (1) for k >= 4 (k = 3: the one-role kernel, two
  // CTAs per SM, measured faster)
  if (s->fused_tc == 3 || (s->fused_tc == 1 && K >= 4)) return launch_fused_tc128_ws_t<K>(s, g, eu, sh, U);
  const size_t smem = (size_t)kTcA * 128 * KR * 2 + (size_t)kTcB * KR * KR * 2;
  static int per_sm_dev[64] = {};   // per device (function attributes are per device)
  const int sdev = s->device;
  int per_sm = sdev >= 0 && sdev < 64 ? per_sm_dev[sdev] : 0;
  if (per_sm == 0) {
    QC_CUDA(cudaFuncSetAttribute(k_fused_tc128<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    QC_CUDA(cudaFuncSetAttribute(k_fused_tc128<K>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared));
    cudaFuncAttributes fa;
    QC_CUDA(cudaFuncGetAttributes(&fa, k_fused_tc128<K>));
    int dev = 0, smem_sm = 0, regs_sm = 0;
    QC_CUDA(cudaGetDevice(&dev));
    QC_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    QC_CUDA(cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev));
    const int warp_regs = ((fa.numRegs * 32 + 255) / 256) * 256;
    constexpr int NT = Tc128Cfg<K>::NT;
    const int by_regs = regs_sm / (warp_regs * (NT / 32));
    const int by_smem = smem_sm / (int)(smem + fa.sharedSizeBytes + 1024);
    const int ncol = kTcLev * KR <= 128 ? 128 : (kTcLev * KR <= 256 ? 256 : 512);
    per_sm = std::max(1, std::min(std::min(by_regs, by_smem), std::min(512 / ncol, 2048 / NT)));
    if (sdev >= 0 && sdev < 64) per_sm_dev[sdev] = per_sm;
  }
  const uint64_t cap = (uint64_t)qc_num_sms() * per_sm;
  const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(g.ntiles, cap));
  k_fused_tc128<K><<<grid, Tc128Cfg<K>::NT, smem, s->stream>>>((double2*)s->ptr, g, U, eu, sh, tc_spin(s));
  QC_LAUNCHED("k_fused_tc128");
  return QC_OK;
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
// (the library does not link the driver library itself)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult qr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &qr) == cudaSuccess &&
        qr == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    else
      cudaGetLastError();
  }
  return fn;
}

#ifndef QC_TC128_TMA_TPR5
#define QC_TC128_TMA_TPR5 4   // threads per group row of the k = 5 kernel (2: 1641 ms, 4: 1611 ms for
                              // the n=30 brickwork at k = 5)
#endif
template <int K> struct Tc128TmaCfg {
  static constexpr int TPR = K == 5 ? QC_TC128_TMA_TPR5 : 2;   // threads per group row
  static constexpr int NT = 128 * TPR;
};

template <int K>
int launch_fused_tc128_tma_t(qc_state* s, const qc_op& op, const GeomF& g, int eu, int sh, const MatC128<K>& U) {
  constexpr int D = 1 << K, KR = 2 * D;
  constexpr int TPR = Tc128TmaCfg<K>::TPR, NT = Tc128TmaCfg<K>::NT;
  auto encode = tensor_map_encoder();
  if (!encode) return qc_fail(QC_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  const uint64_t N = 1ull << s->n;
  const uint32_t L = 1u << g.lb;
  // the state as rows of 128 amplitudes (256 64-bit words); a run of L amplitudes is a box of L / 128 rows
  CUtensorMap map;
  const cuuint64_t gdim[2] = {256, (cuuint64_t)(N / 128)};
  const cuuint64_t gstride[1] = {2048};
  const cuuint32_t box[2] = {256, L / 128};
  const cuuint32_t estr[2] = {1, 1};
  CUresult cr = encode(&map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, s->ptr, gdim, gstride, box, estr,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) return qc_fail(QC_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)cr);
  TmaGeom tg;
  tg.run_rows = L / 128;
  tg.nruns = 1u << g.kh;
  tg.tile_bytes = 128u * D * 16u;
  const size_t xoff = (((size_t)kTcA * 128 * KR * 2 + (size_t)kTcB * KR * KR * 2) + 1023) & ~(size_t)1023;
  const size_t smem = xoff + (size_t)tg.tile_bytes;
  static int per_sm_dev[64] = {};
  const int sdev = s->device;
  int per_sm = sdev >= 0 && sdev < 64 ? per_sm_dev[sdev] : 0;
  if (per_sm == 0) {
    QC_CUDA(cudaFuncSetAttribute(k_fused_tc128_tma<K, TPR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    QC_CUDA(cudaFuncSetAttribute(k_fused_tc128_tma<K, TPR>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared));
    cudaFuncAttributes fa;
    QC_CUDA(cudaFuncGetAttributes(&fa, k_fused_tc128_tma<K, TPR>));
    int dev = 0, smem_sm = 0, regs_sm = 0;
    QC_CUDA(cudaGetDevice(&dev));
    QC_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    QC_CUDA(cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev));
    const int warp_regs = ((fa.numRegs * 32 + 255) / 256) * 256;
    const int by_regs = regs_sm / (warp_regs * (NT / 32));
    const int by_smem = smem_sm / (int)(smem + fa.sharedSizeBytes + 1024);
    const int ncol = kTcLev * KR <= 128 ? 128 : (kTcLev * KR <= 256 ? 256 : 512);
    per_sm = std::max(1, std::min(std::min(by_regs, by_smem), std::min(512 / ncol, 2048 / NT)));
    if (sdev >= 0 && sdev < 64) per_sm_dev[sdev] = per_sm;
  }
  const uint64_t cap = (uint64_t)qc_num_sms() * per_sm;
  const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(g.ntiles, cap));
  k_fused_tc128_tma<K, TPR><<<grid, NT, smem, s->stream>>>((double2*)s->ptr, g, U, eu, sh, tc_spin(s), map, tg);
  QC_LAUNCHED("k_fused_tc128_tma");
  return QC_OK;
}

// complex128 (float-float arithmetic) k = 3..5 blocks with 128-group tiles:
// tensor cores with exact digit slices.
int launch_fused_tc128(qc_state* s, const qc_op& op, bool* done) {
  *done = false;
  if (op.k < 3 || op.k > 5 || s->n - op.k - op.nc < 7) return QC_OK;
  GeomF g;
  size_t smem = 0;
  if (!fused_geom(s, op, 8, g, smem) || g.tg_log != 7) return QC_OK;
  *done = true;
  switch (op.k) {
    case 3: return launch_fused_tc128_t<3>(s, op, g);
    case 4: return launch_fused_tc128_t<4>(s, op, g);
    default: return launch_fused_tc128_t<5>(s, op, g);
  }
}

// complex64 k = 3..5 blocks with 128-group tiles go to the tensor cores.
int launch_fused_tc(qc_state* s, const qc_op& op, bool* done) {
  *done = false;
  if (op.k < 3 || op.k > 5 || s->n - op.k - op.nc < 7) return QC_OK;
  GeomF g;
  size_t smem = 0;
  if (!fused_geom(s, op, 8, g, smem) || g.tg_log != 7) return QC_OK;
  *done = true;
  switch (op.k) {
    case 3: return launch_fused_tc_t<3>(s, op, g);
    case 4: return launch_fused_tc_t<4>(s, op, g);
    default: return launch_fused_tc_t<5>(s, op, g);
  }
}


template <class Ar>
int launch_linear_phase(qc_state* s, const qc_op& op) {
  constexpr int L = Ar::V == 4 ? 2 : 1;
  LinGeom lg;
  std::memset(&lg, 0, sizeof(lg));
  int cpos[1] = {op.anchor}, cval[1] = {1};
  Plan P;
  if (int rc = build_geom(s, L, nullptr, 0, cpos, cval, 1, P)) return rc;
  lg.g = P.g;
  // groups of <= 8 linear bits, in ascending position order
  int order[QC_MAX_LIN];
  for (int i = 0; i < op.nlin; i++) order[i] = i;
  std::sort(order, order + op.nlin, [&](int a, int b) { return op.lin_pos[a] < op.lin_pos[b]; });
  lg.ngroups = (op.nlin + 7) / 8;
  if (lg.ngroups > kLinGroups) return qc_fail(QC_ERR_ARG, "internal: %d linear bits", op.nlin);
  if (lg.ngroups == 0) lg.ngroups = 1;   // theta0 only: a one-entry table
  std::vector<typename Ar::coef_t> tab;
  for (int g = 0; g < lg.ngroups; g++) {
    const int b0 = g * 8, nb = std::min(8, std::max(0, op.nlin - b0));
    lg.gbits[g] = nb;
    lg.toff[g] = (int)tab.size();
    bool contig = true;
    for (int b = 0; b < nb; b++) {
      lg.gpos[g][b] = op.lin_pos[order[b0 + b]];
      if (b > 0 && lg.gpos[g][b] != lg.gpos[g][b - 1] + 1) contig = false;
    }
    lg.gcontig[g] = contig ? 1 : 0;
    if (nb == 0) lg.gpos[g][0] = 0;
    for (int m = 0; m < (1 << nb); m++) {
      double ph = g == 0 ? op.theta0 : 0.0;
      for (int b = 0; b < nb; b++) if ((m >> b) & 1) ph += op.lin_theta[order[b0 + b]];
      tab.push_back(Ar::make_coef(std::cos(ph), std::sin(ph)));
    }
  }
  if (tab.size() > (size_t)kLinTab) return qc_fail(QC_ERR_ARG, "internal: phase table of %zu entries", tab.size());
  LinTab<Ar> T;
  std::memcpy(T.t, tab.data(), tab.size() * sizeof(typename Ar::coef_t));
  k_linear_phase<Ar><<<grid_for(lg.g.ntiles, kThreads), kThreads, 0, s->stream>>>((vec32*)s->ptr, lg, T,
                                                                                  (int)tab.size());
  QC_LAUNCHED("k_linear_phase");
  return QC_OK;
}


// Dense 1-qubit gate on the anchor + linear phase run, one sweep (op.pre = 1).
template <class Ar>
int launch_dense_linphase(qc_state* s, const qc_op& op) {
  if constexpr (std::is_same<Ar, ArC128x>::value) {
    if (s->packed) return launch_dense_linphase<ArC128p>(s, op);
  }
  constexpr int V = Ar::V;
  constexpr int L = V == 4 ? 2 : 1;
  constexpr int R = kDlR;
  constexpr int W = L + 2;                   // window bits: in-vector + log2 R
  static_assert((1 << W) == V * R, "window table size");
  using Hi = typename HiAr<Ar>::type;
  if (op.anchor < W) return qc_fail(QC_ERR_ARG, "internal: merged phase sweep on anchor bit %d", op.anchor);
  DLGeom dg;
  std::memset(&dg, 0, sizeof(dg));
  int tpos[1] = {op.anchor};
  Plan P;
  if (int rc = build_geom(s, L, tpos, 1, nullptr, nullptr, 0, P)) return rc;
  if (P.KH != 1 || P.g.ntiles % R) return qc_fail(QC_ERR_ARG, "internal: merged phase sweep geometry");
  dg.g = P.g;
  auto tab = std::make_unique<DLTab<Ar>>();
  std::memset(tab.get(), 0, sizeof(DLTab<Ar>));
  // window table: theta0 and the linear bits below W
  for (int x = 0; x < V * R; x++) {
    double ph = op.theta0;
    for (int j = 0; j < op.nlin; j++)
      if (op.lin_pos[j] < W && ((x >> op.lin_pos[j]) & 1)) ph += op.lin_theta[j];
    tab->w[x] = Ar::make_coef(std::cos(ph), std::sin(ph));
  }
  // high tables: the linear bits at W and above, <= 8 per table, ascending
  int order[QC_MAX_LIN], nh = 0;
  for (int j = 0; j < op.nlin; j++)
    if (op.lin_pos[j] >= W) order[nh++] = j;
  std::sort(order, order + nh, [&](int a, int b) { return op.lin_pos[a] < op.lin_pos[b]; });
  dg.nhg = (nh + 7) / 8;
  if (dg.nhg > kDlGroups) return qc_fail(QC_ERR_ARG, "internal: %d linear bits", nh);
  int ntab = 0;
  for (int g = 0; g < dg.nhg; g++) {
    const int b0 = g * 8, nb = std::min(8, nh - b0);
    dg.hbits[g] = nb;
    dg.hoff[g] = ntab;
    bool contig = true;
    for (int b = 0; b < nb; b++) {
      dg.hpos[g][b] = op.lin_pos[order[b0 + b]];
      if (b > 0 && dg.hpos[g][b] != dg.hpos[g][b - 1] + 1) contig = false;
    }
    dg.hcontig[g] = contig ? 1 : 0;
    for (int m = 0; m < (1 << nb); m++) {
      double ph = 0.0;
      for (int b = 0; b < nb; b++) if ((m >> b) & 1) ph += op.lin_theta[order[b0 + b]];
      tab->hi[ntab++] = Hi::make_coef(std::cos(ph), std::sin(ph));
    }
  }
  MatD<Ar, 2> M;
  MatD<Hi, 2> Mh;
  for (int i = 0; i < 4; i++) {
    M.m[i] = Ar::make_coef(op.U[2 * i], op.U[2 * i + 1]);
    Mh.m[i] = Hi::make_coef(op.U[2 * i], op.U[2 * i + 1]);
  }
  const uint64_t nruns = P.g.ntiles / R;
  const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((nruns + kThreads - 1) / kThreads,
                                                                   (uint64_t)qc_num_sms() * 8));
  if constexpr (std::is_same<Ar, ArC128p>::value) {
    if (s->packed == 2) {            // fixed-binade chains: exponent offsets of U's rows
      int esr[2];
      for (int r = 0; r < 2; r++) {
        double S = 0.0;
        for (int c = 0; c < 2; c++) S += std::fabs(op.U[2 * (2 * r + c)]) + std::fabs(op.U[2 * (2 * r + c) + 1]);
        esr[r] = S > 0.0 ? (int)std::ceil(std::log2(2.0 * S * (1.0 + 0x1p-10))) : -200;
        if (S > 0.0 && (esr[r] > 100 || esr[r] < -100))
          return qc_fail(QC_ERR_ARG, "matrix entries out of range for the complex128 sweep");
      }
      k_dense_linphase<Ar, R, true><<<grid, kThreads, 0, s->stream>>>((vec32*)s->ptr, dg, M, Mh, *tab, ntab,
                                                                       esr[0], esr[1]);
      QC_LAUNCHED("k_dense_linphase");
      return QC_OK;
    }
  }
  k_dense_linphase<Ar, R><<<grid, kThreads, 0, s->stream>>>((vec32*)s->ptr, dg, M, Mh, *tab, ntab, 0, 0);
  QC_LAUNCHED("k_dense_linphase");
  return QC_OK;
}


// A run of disjoint SWAPs as one bit-permutation sweep (QC_OP_PERMUTE).
template <int E>
int launch_permute(qc_state* s, const qc_op& op) {
  constexpr int VA = 32 / E;
  const int n = s->n;
  int pi[64];
  for (int b = 0; b < n; b++) pi[b] = b;
  for (int i = 0; i < op.nperm; i++) {
    const int a = op.perm_a[i], b = op.perm_b[i];
    if (a < 0 || b < 0 || a >= n || b >= n || a == b || pi[a] != a || pi[b] != b)
      return qc_fail(QC_ERR_ARG, "internal: permutation pairs are not disjoint");
    pi[a] = b;
    pi[b] = a;
  }
  // low bits: segments of 2^5 amplitudes (256 or 512 bytes), at least one vector
  const int t = std::min(n, kPermT);
  if ((1 << t) < VA) return qc_fail(QC_ERR_ARG, "internal: state below one vector");
  uint64_t tmask = (1ull << t) - 1ull;
  for (int b = 0; b < t; b++) tmask |= 1ull << pi[b];
  PermGeom pg;
  std::memset(&pg, 0, sizeof(pg));
  pg.t = t;
  for (int b = t; b < n; b++)
    if ((tmask >> b) & 1) pg.hpos[pg.h++] = b;
  for (int b = 0; b < n; b++)
    if ((tmask >> b) & 1) pg.ins[pg.nins++] = b;
  // outside bits (compressed order) and the pairs among them
  int cidx[64], nO = 0;
  for (int b = 0; b < n; b++) cidx[b] = ((tmask >> b) & 1) ? -1 : nO++;
  for (int b = 0; b < n; b++)
    if (cidx[b] >= 0 && pi[b] > b) { pg.pa[pg.npairs] = cidx[b]; pg.pb[pg.npairs] = cidx[pi[b]]; pg.npairs++; }
  pg.ntiles = 1ull << nO;
  const uint32_t ntile = 1u << (t + pg.h);
  if (ntile > (uint32_t)kPermMaxTile) return qc_fail(QC_ERR_ARG, "internal: permutation tile of %u", ntile);
  // src[u]: local index of the source of output local index u; local index =
  // (high tile bits, in hpos order) << t | low bits
  auto local_to_bits = [&](uint32_t u) {
    uint64_t y = u & ((1u << t) - 1u);
    for (int i = 0; i < pg.h; i++) y |= (uint64_t)((u >> (t + i)) & 1u) << pg.hpos[i];
    return y;
  };
  auto bits_to_local = [&](uint64_t y) {
    uint32_t u = (uint32_t)(y & ((1ull << t) - 1ull));
    for (int i = 0; i < pg.h; i++) u |= (uint32_t)((y >> pg.hpos[i]) & 1ull) << (t + i);
    return u;
  };
  auto tab = std::make_unique<PermTab>();
  for (uint32_t u = 0; u < ntile; u++) {
    const uint64_t y = local_to_bits(u);
    uint64_t x = 0;                            // pi(y) on the tile bits (pi is its own inverse)
    for (int b = 0; b < n; b++)
      if ((tmask >> b) & 1) x |= ((y >> b) & 1ull) << pi[b];
    tab->src[u] = (uint16_t)bits_to_local(x);
  }
  const size_t smem = 4 * (size_t)ntile * E + (size_t)ntile * 2 + 8 + ((size_t)8 << pg.h) +
                      kPermBatch * (8 + 8 + 4) + 4;
  static bool attr[2][64] = {};
  const int dev = s->device;
  if (dev >= 0 && dev < 64 && !attr[E == 16][dev]) {
    QC_CUDA(cudaFuncSetAttribute(k_permute<E>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(4 * (size_t)kPermMaxTile * E + kPermMaxTile * 2 + 8 + (8 << kPermT) +
                                       kPermBatch * 20 + 4)));
    attr[E == 16][dev] = true;
  }
  const uint64_t nbatches = (pg.ntiles + kPermBatch - 1) / kPermBatch;
  const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(nbatches, (uint64_t)qc_num_sms() * 4));
  k_permute<E><<<grid, kThreads, smem, s->stream>>>((vec32*)s->ptr, pg, *tab);
  QC_LAUNCHED("k_permute");
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
    if constexpr (Ar::V == 4) {
      if (s->fused_tc) {
        if (int rc = launch_fused_tc(s, op, &done)) return rc;
        if (done) return QC_OK;
      }
    }
    if constexpr (std::is_same<Ar, ArC128x>::value) {
      if (s->fused_tc) {
        if (int rc = launch_fused_tc128(s, op, &done)) return rc;
        if (done) return QC_OK;
      }
    }
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

int qc_tc_timeouts(int* count) {
  QC_CUDA(cudaMemcpyFromSymbol(count, g_tc_timeouts, sizeof(int)));
  return QC_OK;
}

int qc_take_device_status(const char* where) {
  int count = 0;
  if (int rc = qc_tc_timeouts(&count)) return rc;
  if (count == 0) return QC_OK;
  const int zero = 0;
  QC_CUDA(cudaMemcpyToSymbol(g_tc_timeouts, &zero, sizeof(int)));
  return qc_fail(QC_ERR_TIMEOUT, "%s: %d tensor-core wait(s) on this device gave up; the states they "
                 "were updating are incomplete", where, count);
}

int qc_launch_op(qc_state* s, const qc_op& op) {
  if (op.kind == QC_OP_PERMUTE) {
    if (s->dtype == QC_C64) return launch_permute<8>(s, op);
    return launch_permute<16>(s, op);
  }
  if (op.kind == QC_OP_LINEAR_PHASE && op.pre) {
    if (s->dtype == QC_C64) return launch_dense_linphase<ArC64>(s, op);
    if (s->arith == QC_ARITH_NATIVE) return launch_dense_linphase<ArC128>(s, op);
    return launch_dense_linphase<ArC128x>(s, op);
  }
  if (op.kind == QC_OP_LINEAR_PHASE) {
    if (s->n < 3) return qc_fail(QC_ERR_ARG, "internal: linear phase op on n < 3");
    if (s->dtype == QC_C64) return launch_linear_phase<ArC64>(s, op);
    if (s->arith == QC_ARITH_NATIVE) return launch_linear_phase<ArC128>(s, op);
    return launch_linear_phase<ArC128x>(s, op);
  }
  if (s->dtype == QC_C64) return dispatch<ArC64>(s, op);
  if (s->arith == QC_ARITH_NATIVE) return dispatch<ArC128>(s, op);
  return dispatch<ArC128x>(s, op);
}
