// qc_expect.cu -- <psi| sum_t c_t P_t |psi> for Pauli sums.
//
// For a Pauli string P with flip mask F (its X and Y qubits), phase mask
// Q (its Y and Z qubits) and nY Y factors, P|y> = i^nY (-1)^popc(y & Q) |y^F>
// (X|b> = |1-b>, Y|b> = i(-1)^b |1-b>, Z|b> = (-1)^b |b>), so
//   <psi|P|psi> = sum_y i^nY (-1)^popc(y & Q) conj(psi_{y^F}) psi_y .
// qc_expect evaluates the sum in tiled passes (k_pauli_tile, below): each
// pass covers every term whose flip mask lies in the span of its tile bits.
// qc_expect_noalloc keeps the simpler form, one sweep per distinct flip mask
// (k_pauli_sweep): the sweep visits each pair {y, y^F} once (y with the
// pivot bit of F clear), forms the overlap products and adds every term's
// signed contribution to an FP64 accumulator.  Either way per-block partial
// sums go to device memory and a single-block kernel adds them up in a fixed
// order, so the result is deterministic.
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

// ---------------------------------------------------------------------------
// qc_expect: tiled passes.
//
// A pass reads the state once, one tile at a time.  A tile is a set of 2^L
// basis indices y = base ^ G(hc) ^ low: `low` runs over the m lowest bits,
// hc over h bits that select a combination G(hc) of h generator masks (each
// with its own pivot bit at or above m, no generator containing another's
// pivot), and `base` over the remaining bits (zero at the low and pivot
// bits).  With the local index l = hc << m | low a term with flip mask F maps
// the tile onto itself whenever F lies in the span of the low bits and the
// generators: then y ^ F = base ^ G(hc ^ hc_F) ^ (low ^ F_low), i.e. the local
// index l ^ FL with FL = hc_F << m | F_low.  The sign splits the same way:
// popc(y & Q) = popc(base & Q) + popc(l & QL) (mod 2) with QL = q_hc << m |
// (Q & low mask), bit i of q_hc being the parity of G_i & Q.  So one pass,
// tile by tile in shared memory, evaluates every term whose flip mask lies in
// its span; the host chooses the generators so that few passes cover all
// terms (for nearest-neighbour Hamiltonians on 30 qubits: 4 passes instead of
// one sweep per distinct flip mask).
//
// Arithmetic.  The sweeps run in FP32 error-free transformations (GB300's
// FP64 rate is far below its FP32 rate): amplitudes are split into hi + lo
// floats (complex128: 47 significant bits; complex64: exact), products are
// TwoProduct-exact in their hi * hi part, sums are Knuth TwoSum with the
// rounding errors carried in a lo word, and every block finishes in FP64.
// Pair terms (F != 0): a pair {y, y ^ F} contributes
//   s_y * {2 Re w, -2 Im w, -2 Re w, 2 Im w}[nY mod 4],  w = conj(psi_{y^F}) psi_y,
// (the y ^ F half equals the y half because popc(F & Q) = nY).  Diagonal
// terms: a thread takes 16 amplitudes that differ in four local bits, forms
// the Walsh-Hadamard transform W[u] = sum_j (-1)^popc(j & u) |psi_j|^2 of
// those 16 and reads each term's contribution as +-W[QL restricted to the four
// bits], so the per-term cost is paid once per 16 amplitudes.
namespace {

constexpr int kTileThreads = 256;
constexpr int kTileMaxH = 9;       // generator masks per pass
constexpr int kGroupTerms = 2;     // pair terms evaluated together per flip mask

struct TTerm {                     // one term inside a pass
  uint64_t q;                      // phase mask Q (global bit positions)
  uint32_t ql;                     // local phase mask QL
  uint32_t pad;
  float kh, kh2, kl, kl2;          // weight k (c_t, times +-2 for pair terms) as hi kh + lo kl;
                                   // (kh2, kl2) = +-(kh, kl): the weight of the second lane of a
                                   // packed pair sum, negative when the term weighs Im w
};
static_assert(sizeof(TTerm) == 32, "terms are 32-byte records; the weights are one 16-byte load");
struct TGroup {                    // pair terms sharing one local flip mask
  uint32_t fl;                     // FL
  int pivot;                       // highest set bit of FL
  int t0, nt;                      // terms[t0 .. t0 + nt)
  uint32_t kind;                   // bit 0: the terms weigh Im w (else Re w); bit 1: their
                                   // local phase masks are nonzero (then nt <= kGroupTerms)
};
struct TPass {                     // kernel parameter: one pass
  const TTerm* terms;
  const TGroup* groups;
  uint64_t ntiles;                 // 2^(n - L)
  int m, h, L, wb;                 // low bits, generators, tile bits, WHT window
  int ngroups, dt0, dnt;           // pair groups; diagonal terms [dt0, dt0 + dnt)
  int dtile;                       // the first dtile diagonal terms have QL = 0 (their sign is
                                   // the tile's: the register-resident kernel sums them per tile)
  int piv[kTileMaxH];              // pivot bit of generator i, ascending in i
  uint64_t gen[kTileMaxH];         // generator masks
  int garr[4];                     // register-resident kernel: groups [garr[a], garr[a+1]) (a < 3;
                                   // garr[3] .. ngroups: from shared memory) use arrangement a
  int qmask;                       // bit 4a + b: arrangement a's groups start with the Re-weighted,
                                   // unsigned group of the single register bit b (in order of b)
  int reg;                         // 1: k_pauli_reg (tiles of 2^12), 0: k_pauli_tile
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

// (th, tl) += (kh + kl) * (vh + vl), hi * hi exact, the rest rounded once.
__device__ __forceinline__ void acc_scaled(float& th, float& tl, float kh, float kl, float vh, float vl) {
  const float p = __fmul_rn(kh, vh);
  const float pe = __fmaf_rn(kh, vh, -p);
  const float pl = __fmaf_rn(kh, vl, __fmaf_rn(kl, vh, pe));
  float s, e;
  two_sum(th, p, s, e);
  th = s;
  tl = __fadd_rn(tl, __fadd_rn(e, pl));
}

using P2 = ArC128p;                // packed FP32-pair instructions
// -x per component on the FP32 pipe (0 - x; the sign of a zero does not matter here)
__device__ __forceinline__ uint64_t neg2(uint64_t a) { return P2::sub2(0ull, a); }
// (+-1, +-1) as a packed pair: -1 when `odd` has its lowest bit set
__device__ __forceinline__ uint64_t sgn2(uint32_t odd) {
  const uint32_t f = ((odd & 1u) << 31) | 0x3f800000u;
  return (uint64_t)f | ((uint64_t)f << 32);
}

// Rounded product b * a per component, written as fma(b, a, z) with z a zero
// the compiler cannot see (read from a kernel parameter): a plain multiply
// that feeds the TwoSum below may be fused with its first add by the code
// generator, and TwoSum is not error-free for such a fused sum.
__device__ __forceinline__ uint64_t prod2(uint64_t b, uint64_t a, uint64_t z) { return P2::fma2(b, a, z); }

// Packed TwoSum accumulation: (ah, al) += (p, e) per component.
__device__ __forceinline__ void acc2(uint64_t& ah, uint64_t& al, uint64_t p, uint64_t e) {
  const uint64_t t = P2::add2(ah, p);
  const uint64_t z = P2::sub2(t, ah);
  const uint64_t err = P2::add2(P2::sub2(ah, P2::sub2(t, z)), P2::sub2(p, z));
  ah = t;
  al = P2::add2(al, P2::add2(err, e));
}

// Tile entry: complex128 -> {hi pair (re, im), lo pair (re, im)} (16 bytes);
// complex64 -> the amplitude itself (8 bytes; its lo pair is zero).
template <bool C128> struct TileT;
template <> struct TileT<true> {
  static constexpr int E = 16;     // tile bytes per amplitude
  static constexpr int G = 16;     // state bytes per amplitude
  struct amp { uint64_t h, l; };
  static __device__ __forceinline__ amp get(const unsigned char* t, uint32_t l) {
    const uint4 v = *(const uint4*)(t + (size_t)l * 16);
    return {(uint64_t)v.x | ((uint64_t)v.y << 32), (uint64_t)v.z | ((uint64_t)v.w << 32)};
  }
};
template <> struct TileT<false> {
  static constexpr int E = 8;
  static constexpr int G = 8;
  struct amp { uint64_t h, l; };
  static __device__ __forceinline__ amp get(const unsigned char* t, uint32_t l) {
    return {*(const uint64_t*)(t + (size_t)l * 8), 0ull};
  }
};

// Padded tile layout of the register-resident kernel (below): 16-byte chunk
// c -- amplitude c (complex128) or amplitudes 2c, 2c + 1 (complex64) -- at
// slot c + (c >> 4) (complex128) or c + (c >> 3) (complex64), one spare chunk
// after every 16 (8).  The copy-in, the three arrangements' loads, the
// write-back and the diagonal scratch then touch distinct banks across the
// lanes of a wavefront, and each arrangement's 16 slots of a thread lie at
// constant offsets from a per-thread base (reg_base, reg_stride).
template <bool C128>
__device__ __forceinline__ uint32_t rslot(uint32_t l) {
  const uint32_t c = C128 ? l : (l >> 1);
  return c + (c >> (C128 ? 4 : 3));
}
constexpr uint32_t reg_slots(bool c128) { return c128 ? 4096u + 256u : 2048u + 256u; }   // 16-byte slots per tile

template <bool C128, bool SWZ>
__device__ __forceinline__ typename TileT<C128>::amp tile_get(const unsigned char* t, uint32_t l) {
  if constexpr (!SWZ) {
    return TileT<C128>::get(t, l);
  } else if constexpr (C128) {
    const uint4 v = *(const uint4*)(t + (size_t)rslot<true>(l) * 16);
    return {(uint64_t)v.x | ((uint64_t)v.y << 32), (uint64_t)v.z | ((uint64_t)v.w << 32)};
  } else {
    return {*(const uint64_t*)(t + (size_t)rslot<false>(l) * 16 + (l & 1u) * 8), 0ull};
  }
}

// Load the tile with base index `base` into shared memory: 16-byte
// asynchronous copies (cp.async, no registers held while they are in flight),
// then each thread splits the complex128 entries it copied into hi + lo
// floats in place.  A 16-byte chunk holds one complex128 or two complex64
// amplitudes and never straddles a segment (segments are 2^m >= 2 amplitudes).
template <bool C128>
__device__ __forceinline__ void load_tile(const unsigned char* __restrict__ psi, uint64_t base,
                                          const uint64_t* gtab, const TPass& P, unsigned char* tile) {
  using T = TileT<C128>;
  constexpr int CA = 16 / T::G;                       // amplitudes per chunk
  const uint32_t nchunk = (1u << P.L) / CA;
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(tile);
  const uint32_t lowm = (1u << P.m) - 1u;
  for (uint32_t v = threadIdx.x; v < nchunk; v += kTileThreads) {
    const uint32_t l = v * CA;
    const uint64_t y = (base ^ gtab[l >> P.m]) + (l & lowm);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                 :: "r"(sbase + v * 16u), "l"(psi + y * T::G) : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  if constexpr (C128) {
    for (uint32_t v = threadIdx.x; v < nchunk; v += kTileThreads) {
      uint4* d = (uint4*)(tile + (size_t)v * 16);
      const uint4 x = *d;
      const ArC128x::ff re = ArC128x::split(x.x, x.y);
      const ArC128x::ff im = ArC128x::split(x.z, x.w);
      *d = make_uint4(__float_as_uint(re.h), __float_as_uint(im.h), __float_as_uint(re.l), __float_as_uint(im.l));
    }
  }
}

// Pair terms of one group over the tile; adds their weighted sums to (th, tl).
// IM: the group's terms weigh Im w (odd nY), else Re w.  SIGNED: the terms'
// local phase masks are nonzero (at most kGroupTerms terms, one accumulator
// each); otherwise every term of the group has the same in-tile sum and one
// accumulator serves them all (any number of terms).
template <bool C128, bool IM, bool SIGNED, bool SWZ = false>
__device__ __forceinline__ void tile_group(const unsigned char* tile, const TPass& P, const TGroup& g,
                                           uint64_t base, uint64_t zz, float& th, float& tl) {
  using T = TileT<C128>;
  constexpr int NA = SIGNED ? kGroupTerms : 1;      // accumulators
  uint32_t ql[NA];
#pragma unroll
  for (int k = 0; k < NA; k++) ql[k] = SIGNED ? __ldg(&P.terms[g.t0 + (k < g.nt ? k : 0)].ql) : 0u;
  uint64_t ah[NA], al[NA];
#pragma unroll
  for (int k = 0; k < NA; k++) { ah[k] = 0ull; al[k] = 0ull; }
  const uint32_t npairs = 1u << (P.L - 1);
  const uint32_t hm = ~((1u << g.pivot) - 1u);     // l = j with a zero inserted at the pivot
  // UNR pairs per iteration, their shared-memory loads issued first
  constexpr int UNR = C128 ? 2 : 4;
  const bool full = (npairs & (UNR * kTileThreads - 1)) == 0;
  for (uint32_t j0 = threadIdx.x; j0 < npairs; j0 += UNR * kTileThreads) {
    typename T::amp a[UNR], b[UNR];
    uint32_t l[UNR];
#pragma unroll
    for (int u = 0; u < UNR; u++) {
      uint32_t j = j0 + u * kTileThreads;
      if (!full) j = min(j, npairs - 1u);
      l[u] = j + (j & hm);
      a[u] = tile_get<C128, SWZ>(tile, l[u]);
      b[u] = tile_get<C128, SWZ>(tile, l[u] ^ g.fl);
    }
#pragma unroll
    for (int u = 0; u < UNR; u++) {
      if (!full && j0 + u * kTileThreads >= npairs) break;
      // w = conj(b) a:  Re w = br ar + bi ai (x + y of b*a),  Im w = br ai - bi ar
      // (x - y of b * swap(a)).  Products: hi*hi exact, cross terms rounded.
      const uint64_t ah_ = IM ? P2::swp(a[u].h) : a[u].h;
      // hi*hi products exact (the FMA remainder e), complex128's cross terms rounded;
      // complex64 amplitudes are their hi pairs (lo zero), so its products are exact
      const uint64_t p = prod2(b[u].h, ah_, zz);
      uint64_t e = P2::fma2(b[u].h, ah_, neg2(p));
      if constexpr (C128) {
        const uint64_t al_ = IM ? P2::swp(a[u].l) : a[u].l;
        e = P2::add2(e, P2::fma2(b[u].h, al_, P2::mul2(b[u].l, ah_)));
      }
      if constexpr (SIGNED) {
#pragma unroll
        for (int k = 0; k < NA; k++) {
          if (k < g.nt) {
            const uint64_t sg = sgn2(__popc(l[u] & ql[k]));
            acc2(ah[k], al[k], P2::mul2(p, sg), P2::mul2(e, sg));
          }
        }
      } else {
        acc2(ah[0], al[0], p, e);
      }
    }
  }
  // value = x + y (Re) or x - y (Im) of the packed sums
  float vh[NA], vl[NA];
#pragma unroll
  for (int k = 0; k < NA; k++) {
    const float hx = P2::lo32(ah[k]), lx = P2::lo32(al[k]);
    const float hy = IM ? -P2::hi32(ah[k]) : P2::hi32(ah[k]);
    const float ly = IM ? -P2::hi32(al[k]) : P2::hi32(al[k]);
    float ve;
    two_sum(hx, hy, vh[k], ve);
    vl[k] = __fadd_rn(ve, __fadd_rn(lx, ly));
  }
  static_assert(kGroupTerms == 2, "the selects below pick one of two accumulators");
  for (int k = 0; k < g.nt; k++) {
    const TTerm* tt = &P.terms[g.t0 + k];
    const float xh = (SIGNED && k == 1) ? vh[NA - 1] : vh[0];
    const float xl = (SIGNED && k == 1) ? vl[NA - 1] : vl[0];
    const bool neg = __popcll(base & __ldg(&tt->q)) & 1;
    acc_scaled(th, tl, __ldg(&tt->kh), __ldg(&tt->kl), neg ? -xh : xh, neg ? -xl : xl);
  }
}

// Diagonal terms over the tile (after the pair groups: overwrites the tile).
template <bool C128>
__device__ __forceinline__ void tile_diag(unsigned char* tile, const uint64_t* gtab, const TPass& P, uint64_t base,
                                          uint64_t zz, float& th, float& tl) {
  using T = TileT<C128>;
  const uint32_t ntile = 1u << P.L;
  const uint32_t nchunks = ntile >= 16 ? ntile >> 4 : 1u;
  const int wb = P.wb;
  for (uint32_t c = threadIdx.x; c < nchunks; c += kTileThreads) {
    // chunk start: c deposited into the local bits outside [wb, wb + 4)
    const uint32_t start = (c & ((1u << wb) - 1u)) | ((c >> wb) << (wb + 4));
    float ph[16], pl[16];
#pragma unroll
    for (int k = 0; k < 16; k++) {
      const uint32_t l = start + ((uint32_t)k << wb);
      ph[k] = 0.f;
      pl[k] = 0.f;
      if (l < ntile) {
        const typename T::amp a = T::get(tile, l);
        const uint64_t p = prod2(a.h, a.h, zz);
        // |a|^2 = re^2 + im^2: hi*hi exact (TwoProduct), complex128's 2 hi*lo rounded
        uint64_t e = P2::fma2(a.h, a.h, neg2(p));
        if constexpr (C128) e = P2::add2(e, P2::mul2(P2::add2(a.h, a.h), a.l));
        float s, r;
        two_sum(P2::lo32(p), P2::hi32(p), s, r);
        ph[k] = s;
        pl[k] = __fadd_rn(r, __fadd_rn(P2::lo32(e), P2::hi32(e)));
      }
    }
    // in-register Walsh-Hadamard transform over the 16 entries
#pragma unroll
    for (int b = 1; b < 16; b <<= 1) {
#pragma unroll
      for (int k = 0; k < 16; k++) {
        if (!(k & b)) {
          const float xh = ph[k], xl = pl[k], yh = ph[k | b], yl = pl[k | b];
          float s, e;
          two_sum(xh, yh, s, e);
          ph[k] = s;
          pl[k] = __fadd_rn(__fadd_rn(xl, yl), e);
          two_sum(xh, -yh, s, e);
          ph[k | b] = s;
          pl[k | b] = __fadd_rn(__fsub_rn(xl, yl), e);
        }
      }
    }
    // W[u] replaces entry u of the chunk (each thread reads back only its own)
#pragma unroll
    for (int k = 0; k < 16; k++) {
      const uint32_t l = start + ((uint32_t)k << wb);
      if (l < ntile || k == 0) *(float2*)(tile + (size_t)l * T::E) = make_float2(ph[k], pl[k]);
    }
    // global index of the chunk's first entry: base ^ G(hc) ^ low
    const uint64_t y0 = base ^ gtab[start >> P.m] ^ (start & ((1u << P.m) - 1u));
    constexpr int TU = 4;          // terms per iteration, their loads issued first
    for (int t0 = P.dt0; t0 < P.dt0 + P.dnt; t0 += TU) {
      uint32_t qlt[TU];
      uint64_t qt[TU];
      float kh[TU], kl[TU];
#pragma unroll
      for (int i = 0; i < TU; i++) {
        const TTerm* tt = &P.terms[min(t0 + i, P.dt0 + P.dnt - 1)];
        qlt[i] = __ldg(&tt->ql);
        qt[i] = __ldg(&tt->q);
        kh[i] = __ldg(&tt->kh);
        kl[i] = __ldg(&tt->kl);
      }
      float2 w[TU];
#pragma unroll
      for (int i = 0; i < TU; i++) {
        const uint32_t u = (qlt[i] >> wb) & 15u;
        w[i] = *(const float2*)(tile + (size_t)(start + (u << wb)) * T::E);
      }
#pragma unroll
      for (int i = 0; i < TU; i++) {
        if (t0 + i < P.dt0 + P.dnt) {
          // sign (-1)^popc(y0 & Q) of the chunk's first index y0, folded into the weight
          const uint32_t sb = (uint32_t)__popcll(y0 & qt[i]) << 31;
          acc_scaled(th, tl, __uint_as_float(__float_as_uint(kh[i]) ^ sb),
                     __uint_as_float(__float_as_uint(kl[i]) ^ sb), w[i].x, w[i].y);
        }
      }
    }
  }
}

template <bool C128>
__global__ void __launch_bounds__(kTileThreads, 3)
k_pauli_tile(const unsigned char* __restrict__ psi, const __grid_constant__ TPass P, double* __restrict__ partial) {
  extern __shared__ __align__(16) unsigned char tsm[];
  using T = TileT<C128>;
  unsigned char* tile = tsm;
  uint64_t* gtab = (uint64_t*)(tsm + ((size_t)T::E << P.L));
  for (int c = threadIdx.x; c < (1 << P.h); c += kTileThreads) {
    uint64_t g = 0;
    for (int i = 0; i < P.h; i++)
      if ((c >> i) & 1) g ^= P.gen[i];
    gtab[c] = g;
  }
  const uint64_t zz = P.ntiles >> 63;   // 0 (ntiles <= 2^36), opaque to the compiler
  // A tile's terms are summed in float-float (th, tl); each tile's sum then
  // joins a per-thread FP64 total.  (Carrying one float-float pair across
  // all of a thread's tiles -- hundreds of tiles and tens of thousands of
  // additions at 30 qubits -- let its unnormalised low word lose precision:
  // 3e-10 off a closed form.)
  double tot = 0.0;
  for (uint64_t tix = blockIdx.x; tix < P.ntiles; tix += gridDim.x) {
    float th = 0.f, tl = 0.f;
    uint64_t base = tix << P.m;
    for (int i = 0; i < P.h; i++) base = qc_insert_zero(base, P.piv[i]);
    __syncthreads();                 // previous tile consumed, gtab written
    load_tile<C128>(psi, base, gtab, P, tile);
    __syncthreads();
    for (int gi = 0; gi < P.ngroups; gi++) {
      TGroup g;
      g.fl = __ldg(&P.groups[gi].fl);
      g.pivot = __ldg(&P.groups[gi].pivot);
      g.t0 = __ldg(&P.groups[gi].t0);
      g.nt = __ldg(&P.groups[gi].nt);
      g.kind = __ldg(&P.groups[gi].kind);
      switch (g.kind) {
        case 0: tile_group<C128, false, false>(tile, P, g, base, zz, th, tl); break;
        case 1: tile_group<C128, true, false>(tile, P, g, base, zz, th, tl); break;
        case 2: tile_group<C128, false, true>(tile, P, g, base, zz, th, tl); break;
        default: tile_group<C128, true, true>(tile, P, g, base, zz, th, tl); break;
      }
    }
    if (P.dnt > 0) {
      __syncthreads();               // pair groups done reading the tile
      tile_diag<C128>(tile, gtab, P, base, zz, th, tl);
    }
    tot += ArC128x::f2d(th) + ArC128x::f2d(tl);   // exact conversions (integer operations)
  }
  const double bs = block_sum(tot);
  if (threadIdx.x == 0) partial[blockIdx.x] = bs;
}

// ---- register-resident passes ---------------------------------------------
// Tiles of 2^12 amplitudes, 256 threads.  Each thread holds 16 amplitudes of
// the tile in registers: those whose local index differs only in four
// "register bits".  Three arrangements put the local bits [0, 4), [4, 8) and
// [8, 12) in registers in turn; the tile passes through shared memory between
// them in a swizzled layout (rslot) that keeps every one of these accesses
// free of bank conflicts.  A pair term whose local flip mask FL lies within
// the register bits of an arrangement pairs amplitudes held by one thread, so
// the term costs no shared-memory traffic at all; other pair terms read the
// tile from shared memory as in k_pauli_tile.  Diagonal terms use the
// Walsh-Hadamard transform of the 16 |psi|^2 of arrangement 0.
//
// complex128 pair sums run in a fixed-binade chain instead of float-float
// TwoSum steps: with sigma = 1.5 * 2^E and 2^E at least four times the largest
// possible partial sum, t = fma(b, a, t) stays in [2^E, 2^(E+1)), so t - t'
// is exact (Sterbenz) and the product's remainder fma(b, a, t - t') is the
// rounding error of the step (exact up to 2^-24 of itself); the remainders and
// the hi*lo cross terms add up in a second word.  Three instructions per
// product instead of eight; the in-tile sum is (t - sigma) + lo.
constexpr int kRegL = 12;

__device__ __forceinline__ uint32_t sgn_bits(uint32_t odd) { return (odd & 1u) << 31; }

// sigma (packed twice) for 8 products of amplitudes whose components are at most mx
__device__ __forceinline__ uint64_t chain_sigma(float mx) {
  const int ef = (int)((__float_as_uint(mx) >> 23) & 0xFFu);
  int e = 2 * ef - 120;                  // 2^(e-127) >= 32 mx^2
  e = e < 24 ? 24 : (e > 254 ? 254 : e);
  const uint32_t sg = ((uint32_t)e << 23) | 0x00400000u;
  return (uint64_t)sg | ((uint64_t)sg << 32);
}

// One group of pair terms over the 16 register amplitudes (register bits of
// the current arrangement, the group's flip mask FLR in them).  lsign[k]: the
// parity of the thread's fixed local bits & QL of term k; qlr[k]: QL restricted
// to the register bits.  Per accumulator k the result is the packed pair of
// lane sums: vh[k] (exact, a multiple of ulp(sigma)) + vl[k] (remainders and
// cross terms); lane x holds the sum of br ar (IM: br ai), lane y of bi ai
// (IM: bi ar), so Re w = x + y and Im w = x - y -- the term's packed weight
// (k, +-k) takes that sign.
template <bool C128, int FLR, bool IM, bool SIGNED>
__device__ __forceinline__ void reg_pairs(const uint64_t* ah, const uint64_t* al, uint64_t sig, const uint32_t* lsign,
                                          const uint32_t* qlr, int nt, uint64_t* vh, uint64_t* vl) {
  constexpr int NA = SIGNED ? kGroupTerms : 1;
  constexpr int PIV = FLR >= 8 ? 8 : (FLR >= 4 ? 4 : (FLR >= 2 ? 2 : 1));
  // two independent chains per accumulator (alternate pairs): twice the
  // instruction-level parallelism of one serial chain
  uint64_t t[2][NA], lo[2][NA];
#pragma unroll
  for (int c = 0; c < 2; c++)
#pragma unroll
    for (int k = 0; k < NA; k++) { t[c][k] = sig; lo[c][k] = 0ull; }
  int npair = 0;
#pragma unroll
  for (int r = 0; r < 16; r++) {
    if (r & PIV) continue;
    const int ch = (npair++) & 1;          // compile-time after unrolling
    const int p = r ^ FLR;                 // partner: conj(psi_{y ^ F}) psi_y
    const uint64_t ahp = IM ? P2::swp(ah[r]) : ah[r];
#pragma unroll
    for (int k = 0; k < NA; k++) {
      if (SIGNED && k >= nt) break;
      uint64_t bh = ah[p];
      if constexpr (SIGNED) {
        const uint32_t sb = sgn_bits(lsign[k] ^ (uint32_t)__popc((uint32_t)r & qlr[k]));
        bh ^= (uint64_t)sb | ((uint64_t)sb << 32);
      }
      if constexpr (C128) {
        const uint64_t alp = IM ? P2::swp(al[r]) : al[r];
        uint64_t bl = al[p];
        if constexpr (SIGNED) {
          const uint32_t sb = sgn_bits(lsign[k] ^ (uint32_t)__popc((uint32_t)r & qlr[k]));
          bl ^= (uint64_t)sb | ((uint64_t)sb << 32);
        }
        const uint64_t t1 = P2::fma2(bh, ahp, t[ch][k]);
        const uint64_t rr = P2::fma2(bh, ahp, P2::sub2(t[ch][k], t1));
        t[ch][k] = t1;
        lo[ch][k] = P2::fma2(bl, ahp, P2::fma2(bh, alp, P2::add2(lo[ch][k], rr)));
      } else {
        // complex64: the same chain without lo parts (exact products, float-float sums)
        const uint64_t t1 = P2::fma2(bh, ahp, t[ch][k]);
        const uint64_t rr = P2::fma2(bh, ahp, P2::sub2(t[ch][k], t1));
        t[ch][k] = t1;
        lo[ch][k] = P2::add2(lo[ch][k], rr);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < NA; k++) {
    // (t0 - sigma) + (t1 - sigma): multiples of ulp(sigma) below 2^(E-2) each, so exact
    vh[k] = P2::add2(P2::sub2(t[0][k], sig), P2::sub2(t[1][k], sig));
    vl[k] = P2::add2(lo[0][k], lo[1][k]);
  }
}

// Packed weighted accumulation, per lane: (TH, TL) += (wh + wl) * (xh + xl),
// wh * xh exact (TwoProduct), the cross terms rounded once, the sum TwoSum.
__device__ __forceinline__ void acc_w2(uint64_t& TH, uint64_t& TL, uint64_t wh, uint64_t wl, uint64_t xh, uint64_t xl,
                                       uint64_t zz) {
  const uint64_t p = prod2(wh, xh, zz);
  const uint64_t e = P2::fma2(wh, xh, neg2(p));
  acc2(TH, TL, p, P2::fma2(wh, xl, P2::fma2(wl, xh, e)));
}

// Pair groups staged in shared memory (the first kRegGroupSmem of a pass's
// register-arrangement groups): the record once per CTA, the weights once
// per tile (warp 0, while the tile copy is in flight).
constexpr int kRegGroupSmem = 128;
struct RegGroup {
  uint32_t fl, kind;
  int t0, nt;
  uint32_t ql0, ql1;               // the local phase masks of a signed group's (at most two) terms
  uint32_t pad[2];
};
struct RegGW {                     // packed weights (hi, lo), each lane pair (k, +-k)
  uint64_t wh0, wl0;               // unsigned group: sum_t c_t (-1)^popc(base & Q_t); signed: term 0's
  uint64_t wh1, wl1;               // signed group: term 1's
};

// Packed weights of term t, its sign (-1)^popc(base & Q_t) applied.
__device__ __forceinline__ void term_w2(const TTerm* tt, uint64_t base, uint64_t& wh, uint64_t& wl) {
  const uint4 w = __ldg((const uint4*)&tt->kh);                  // kh, kh2, kl, kl2
  const uint64_t sb = (uint64_t)(__popcll(base & __ldg(&tt->q)) & 1) << 31;
  const uint64_t s2 = sb | (sb << 32);
  wh = ((uint64_t)w.x | ((uint64_t)w.y << 32)) ^ s2;
  wl = ((uint64_t)w.z | ((uint64_t)w.w << 32)) ^ s2;
}

// The groups [g0, g1) of arrangement `a` (register bits [4a, 4a + 4)) for this
// thread's registers; lbase = the thread's local index with zero register bits.
// Each term (an unsigned group: its terms' summed weight) adds its packed
// weight times the group's packed lane sums to the packed accumulator
// (TH, TL); the lanes are added once per tile.
template <bool C128>
__device__ __forceinline__ void reg_groups(const TPass& P, const RegGroup* sg, const RegGW* sw, int g0, int g1, int a,
                                           uint32_t lbase, uint64_t base, const uint64_t* ah, const uint64_t* al,
                                           uint64_t sig, uint64_t zz, uint64_t& TH, uint64_t& TL) {
  // weight of an unsigned group (staged, or summed from its terms) times its lane sums
  auto weigh = [&](int gi, uint64_t xh, uint64_t xl) {
    if (gi < kRegGroupSmem) {
      const uint4 w0 = *(const uint4*)&sw[gi].wh0;
      acc_w2(TH, TL, (uint64_t)w0.x | ((uint64_t)w0.y << 32), (uint64_t)w0.z | ((uint64_t)w0.w << 32), xh, xl, zz);
    } else {
      const int t0 = __ldg(&P.groups[gi].t0), nt = __ldg(&P.groups[gi].nt);
      for (int k = 0; k < nt; k++) {
        uint64_t wh, wl;
        term_w2(&P.terms[t0 + k], base, wh, wl);
        acc_w2(TH, TL, wh, wl, xh, xl, zz);
      }
    }
  };
  // The arrangement's Re-weighted unsigned groups of single register bits
  // (X or Y on one qubit, ...) come first: no dispatch, and with all four
  // present one straight run of four chains that the compiler interleaves.
  const uint32_t qm = ((uint32_t)P.qmask >> (4 * a)) & 15u;
  int g = g0;
  if (qm == 15u) {
    const uint32_t z2[2] = {0u, 0u};
    uint64_t h1[2], l1[2], h2[2], l2[2], h4[2], l4[2], h8[2], l8[2];
    reg_pairs<C128, 1, false, false>(ah, al, sig, z2, z2, 1, h1, l1);
    reg_pairs<C128, 2, false, false>(ah, al, sig, z2, z2, 1, h2, l2);
    reg_pairs<C128, 4, false, false>(ah, al, sig, z2, z2, 1, h4, l4);
    reg_pairs<C128, 8, false, false>(ah, al, sig, z2, z2, 1, h8, l8);
    weigh(g, h1[0], l1[0]);
    weigh(g + 1, h2[0], l2[0]);
    weigh(g + 2, h4[0], l4[0]);
    weigh(g + 3, h8[0], l8[0]);
    g += 4;
  } else if (qm) {
    const uint32_t z2[2] = {0u, 0u};
    uint64_t vh1[2], vl1[2];
    if (qm & 1u) { reg_pairs<C128, 1, false, false>(ah, al, sig, z2, z2, 1, vh1, vl1); weigh(g++, vh1[0], vl1[0]); }
    if (qm & 2u) { reg_pairs<C128, 2, false, false>(ah, al, sig, z2, z2, 1, vh1, vl1); weigh(g++, vh1[0], vl1[0]); }
    if (qm & 4u) { reg_pairs<C128, 4, false, false>(ah, al, sig, z2, z2, 1, vh1, vl1); weigh(g++, vh1[0], vl1[0]); }
    if (qm & 8u) { reg_pairs<C128, 8, false, false>(ah, al, sig, z2, z2, 1, vh1, vl1); weigh(g++, vh1[0], vl1[0]); }
  }
  for (int gi = g; gi < g1; gi++) {
    const bool staged = gi < kRegGroupSmem;
    uint32_t fl, kind, ql0 = 0u, ql1 = 0u;
    int t0, nt;
    if (staged) {
      const uint4 r = *(const uint4*)&sg[gi];
      fl = r.x; kind = r.y; t0 = (int)r.z; nt = (int)r.w;
      if (kind & 2u) {
        const uint2 q = *(const uint2*)&sg[gi].ql0;
        ql0 = q.x; ql1 = q.y;
      }
    } else {
      fl = __ldg(&P.groups[gi].fl);
      t0 = __ldg(&P.groups[gi].t0);
      nt = __ldg(&P.groups[gi].nt);
      kind = __ldg(&P.groups[gi].kind);
      if (kind & 2u) {
        ql0 = __ldg(&P.terms[t0].ql);
        if (nt > 1) ql1 = __ldg(&P.terms[t0 + 1].ql);
      }
    }
    static_assert(kGroupTerms == 2, "two accumulators per signed group");
    uint32_t lsign[kGroupTerms] = {0u, 0u}, qlr[kGroupTerms] = {0u, 0u};
    if (kind & 2u) {
      lsign[0] = (uint32_t)__popc(lbase & ql0) & 1u;
      qlr[0] = (ql0 >> (4 * a)) & 15u;
      lsign[1] = (uint32_t)__popc(lbase & ql1) & 1u;
      qlr[1] = (ql1 >> (4 * a)) & 15u;
    }
    uint64_t vh[kGroupTerms] = {0ull, 0ull}, vl[kGroupTerms] = {0ull, 0ull};
    // one jump on (flip mask in the register bits, kind)
    switch ((((fl >> (4 * a)) & 15u) << 2) | kind) {
#define QC_REG_CASE(F)                                                                                 \
  case 4 * F + 0: reg_pairs<C128, F, false, false>(ah, al, sig, lsign, qlr, nt, vh, vl); break;      \
  case 4 * F + 1: reg_pairs<C128, F, true, false>(ah, al, sig, lsign, qlr, nt, vh, vl); break;       \
  case 4 * F + 2: reg_pairs<C128, F, false, true>(ah, al, sig, lsign, qlr, nt, vh, vl); break;       \
  case 4 * F + 3: reg_pairs<C128, F, true, true>(ah, al, sig, lsign, qlr, nt, vh, vl); break;
      QC_REG_CASE(1) QC_REG_CASE(2) QC_REG_CASE(3) QC_REG_CASE(4) QC_REG_CASE(5) QC_REG_CASE(6) QC_REG_CASE(7)
      QC_REG_CASE(8) QC_REG_CASE(9) QC_REG_CASE(10) QC_REG_CASE(11) QC_REG_CASE(12) QC_REG_CASE(13)
      QC_REG_CASE(14) QC_REG_CASE(15)
#undef QC_REG_CASE
      default: break;
    }
    const bool signed_ = (kind & 2u) != 0;
    if (staged) {
      const RegGW* w = &sw[gi];
      const uint4 w0 = *(const uint4*)&w->wh0;
      acc_w2(TH, TL, (uint64_t)w0.x | ((uint64_t)w0.y << 32), (uint64_t)w0.z | ((uint64_t)w0.w << 32), vh[0], vl[0], zz);
      if (signed_ && nt > 1) {
        const uint4 w1 = *(const uint4*)&w->wh1;
        acc_w2(TH, TL, (uint64_t)w1.x | ((uint64_t)w1.y << 32), (uint64_t)w1.z | ((uint64_t)w1.w << 32), vh[1], vl[1],
               zz);
      }
    } else {
      for (int k = 0; k < nt; k++) {
        uint64_t wh, wl;
        term_w2(&P.terms[t0 + k], base, wh, wl);
        const bool second = signed_ && k == 1;
        acc_w2(TH, TL, wh, wl, second ? vh[1] : vh[0], second ? vl[1] : vl[0], zz);
      }
    }
  }
}

// complex128 component (IEEE double: low word w0, high word w1) -> hi + lo
// floats holding its leading 24 and next 23 significand bits (truncated:
// |x - (hi + lo)| < 2^-46 |x|).  |x| below 2^-100 (zero included) is first
// raised to 2^-100 times its significand, sign kept: an absolute change below
// 2^-99 per component, far under the sums' rounding.  |x| < 2^127.
// Fewer instructions than the rounding, flushing split of the gate kernels;
// in an expectation value the truncation costs at most
// 2^-45 * ||psi||^2 * sum |c_t|.
struct ffp { float h, l; };
__device__ __forceinline__ ffp split_tr(uint32_t w0, uint32_t w1) {
  const uint32_t mag = max(w1 & 0x7FFFFFFFu, 0x39B00000u);                 // exponent >= -100
  // rebias the exponent (1023 -> 127), keep 23 mantissa bits; bit 31 of the
  // shifted word is zero for |x| < 2^127, so the sign is or-ed in
  const uint32_t hb = __funnelshift_l(w0, mag - 0x38000000u, 3) | (w1 & 0x80000000u);
  // lo = (b + m) - b with b = +-2^(E-23) (hi's sign and exponent E) and m the
  // next 23 bits (w0 bits 28..6) in b's mantissa field: exact
  const uint32_t b = (hb & 0xFF800000u) - 0x0B800000u;
  const uint32_t lb = b | ((w0 >> 6) & 0x007FFFFFu);
  return {__uint_as_float(hb), __uint_as_float(lb) - __uint_as_float(b)};
}

// Byte offset of thread t's first amplitude of arrangement a in the padded
// tile, and the step between its 16 amplitudes (register bit r at base + r
// stride; complex64 arrangement 0: chunk j of 8 at base + 16 j).
//   complex128: a=0 slot 17t + r; a=1 (t & 15) + 272 (t >> 4) + 17r;
//               a=2 t + (t >> 4) + 272r
//   complex64 (slot of chunk l >> 1, 8 bytes per amplitude): a=0 9t + j;
//               a=1 ((t & 15) >> 1) + 144 (t >> 4) + 9r; a=2 (t >> 1) + (t >> 4) + 144r
template <bool C128>
__device__ __forceinline__ uint32_t reg_base(int a, uint32_t t) {
  if constexpr (C128) {
    return 16u * (a == 0 ? 17u * t : a == 1 ? (t & 15u) + 272u * (t >> 4) : t + (t >> 4));
  } else {
    const uint32_t half = 8u * (t & 1u);
    return a == 0 ? 144u * t
                  : (a == 1 ? 16u * (((t & 15u) >> 1) + 144u * (t >> 4)) + half : 16u * ((t >> 1) + (t >> 4)) + half);
  }
}
template <bool C128>
constexpr uint32_t reg_stride(int a) {
  return C128 ? (a == 0 ? 16u : a == 1 ? 272u : 4352u) : (a == 0 ? 16u : a == 1 ? 144u : 2304u);
}

// Load the 16 register amplitudes of arrangement a (complex128: the split form
// (hi pair, lo pair) from shared memory; RAW: the raw doubles, split here).
template <bool C128, bool RAW>
__device__ __forceinline__ void reg_load(const unsigned char* tile, int a, uint32_t t, uint64_t* ah, uint64_t* al) {
  const unsigned char* b = tile + reg_base<C128>(a, t);
  if (!C128 && a == 0) {
    // complex64, register bits [0, 4): the thread's 8 chunks, 16 bytes each
#pragma unroll
    for (int k = 0; k < 8; k++) {
      const uint4 v = *(const uint4*)(b + 16 * k);
      ah[2 * k] = (uint64_t)v.x | ((uint64_t)v.y << 32);
      ah[2 * k + 1] = (uint64_t)v.z | ((uint64_t)v.w << 32);
      al[2 * k] = al[2 * k + 1] = 0ull;
    }
    return;
  }
  const uint32_t stp = a == 0 ? reg_stride<C128>(0) : a == 1 ? reg_stride<C128>(1) : reg_stride<C128>(2);
#pragma unroll
  for (int r = 0; r < 16; r++) {
    if constexpr (C128) {
      const uint4 v = *(const uint4*)(b + stp * (uint32_t)r);
      if constexpr (RAW) {
        const ffp re = split_tr(v.x, v.y);
        const ffp im = split_tr(v.z, v.w);
        ah[r] = P2::pk(re.h, im.h);
        al[r] = P2::pk(re.l, im.l);
      } else {
        ah[r] = (uint64_t)v.x | ((uint64_t)v.y << 32);
        al[r] = (uint64_t)v.z | ((uint64_t)v.w << 32);
      }
    } else {
      ah[r] = *(const uint64_t*)(b + stp * (uint32_t)r);
      al[r] = 0ull;
    }
  }
}

// three-input maximum (sm_100 and later)
__device__ __forceinline__ float fmax3(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

// largest |component| (hi parts) of the 16 register amplitudes
// (four independent maxima, then combined: a quarter of the serial dependence)
__device__ __forceinline__ float reg_max(const uint64_t* ah) {
  float m[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int r = 0; r < 16; r++) m[r & 3] = fmax3(m[r & 3], fabsf(P2::lo32(ah[r])), fabsf(P2::hi32(ah[r])));
  return fmax3(fmaxf(m[0], m[1]), m[2], m[3]);
}

// CTAs per SM of k_pauli_reg (its register bound: 128 / 85 registers a thread)
constexpr int reg_ctas_per_sm(bool c128) { return c128 ? 2 : 3; }

// Tiles of the register-resident kernel: 3 low bits, 9 generators.
constexpr int kRegM = 3;
constexpr int kRegH = kRegL - kRegM;
// Diagonal terms with QL != 0 whose base-signed weights a tile stages in
// shared memory (further ones take their sign and weight per thread).
constexpr int kRegDiagSmem = 256;

// Per-tile values staged in shared memory by warp 0.
struct RegMisc {
  uint64_t base[2];                // tile bases, double-buffered (next tile's written during this one)
  float kh, kl;                    // sum over the QL = 0 diagonal terms of c_t (-1)^popc(base & Q_t)
  uint32_t pad[2];
};
struct RegDiag {                   // a QL != 0 diagonal term, weight signed by the tile base
  float kh, kl;
  uint32_t ql, pad;
};

// Index of the first amplitude of tile tix: tix << m with zeros inserted at
// the generators' pivot bits (ascending).
__device__ __forceinline__ uint64_t tile_base(const TPass& P, uint64_t tix) {
  uint64_t b = tix << P.m;
  for (int i = 0; i < P.h; i++) b = qc_insert_zero(b, P.piv[i]);
  return b;
}

template <bool C128>
__global__ void __launch_bounds__(kTileThreads, reg_ctas_per_sm(C128))
k_pauli_reg(const unsigned char* __restrict__ psi, const __grid_constant__ TPass P, double* __restrict__ partial) {
  extern __shared__ __align__(16) unsigned char rsm[];
  constexpr uint32_t kChunks = C128 ? (1u << kRegL) : (1u << (kRegL - 1));   // 16-byte chunks per tile
  constexpr uint32_t kG = C128 ? 16u : 8u;                                    // state bytes per amplitude
  constexpr int kNC = (int)(kChunks / kTileThreads);                         // chunks per thread
  unsigned char* tile = rsm;
  uint64_t* gtab = (uint64_t*)(rsm + (size_t)reg_slots(C128) * 16);   // byte offsets of the generator combinations
  RegMisc* misc = (RegMisc*)(gtab + (1 << kRegH));
  const int ngs = P.garr[3] < kRegGroupSmem ? P.garr[3] : kRegGroupSmem;   // staged pair groups
  RegGroup* sg = (RegGroup*)(misc + 1);
  RegGW* sw = (RegGW*)(sg + ngs);
  RegDiag* drec = (RegDiag*)(sw + ngs);
  const uint32_t t = threadIdx.x;
  for (int gi = (int)t; gi < ngs; gi += kTileThreads) {
    RegGroup g;
    g.fl = __ldg(&P.groups[gi].fl);
    g.kind = __ldg(&P.groups[gi].kind);
    g.t0 = __ldg(&P.groups[gi].t0);
    g.nt = __ldg(&P.groups[gi].nt);
    g.ql0 = (g.kind & 2u) ? __ldg(&P.terms[g.t0].ql) : 0u;
    g.ql1 = ((g.kind & 2u) && g.nt > 1) ? __ldg(&P.terms[g.t0 + 1].ql) : 0u;
    g.pad[0] = g.pad[1] = 0u;
    sg[gi] = g;
  }
  for (int c = (int)t; c < (1 << kRegH); c += kTileThreads) {
    uint64_t g = 0;
    for (int i = 0; i < kRegH; i++)
      if ((c >> i) & 1) g ^= P.gen[i];
    gtab[c] = g * kG;
  }
  if (t == 0) misc->base[0] = tile_base(P, blockIdx.x);
  const uint64_t zz = P.ntiles >> 63;
  const uint32_t lb0 = t << 4;                                   // arrangement 0: bits [0, 4) in registers
  const uint32_t lb1 = (t & 15u) | ((t >> 4) << 8);              // arrangement 1: bits [4, 8)
  const uint32_t lb2 = t & 255u;                                 // arrangement 2: bits [8, 12)
  // Tile copy: this thread's chunk i is chunk v = t + 256 i of the tile, local
  // amplitude l = v (complex128) or 2 v (complex64): generator combination
  // l >> 3 = gi0 + kGiStep * i, low bits l & 7 (lowb in bytes), swizzled slot
  // rslot = v + (v >> 4) = t + (t >> 4) + 272 i (complex128) or
  // v + (v >> 3) = t + (t >> 3) + 288 i (complex64).
  const uint32_t sdst = (uint32_t)__cvta_generic_to_shared(tile) + 16u * (C128 ? t + (t >> 4) : t + (t >> 3));
  constexpr uint32_t kDstStep = C128 ? 16u * 272u : 16u * 288u;
  const uint32_t gi0 = C128 ? (t >> 3) : (t >> 2);
  constexpr uint32_t kGiStep = C128 ? 32u : 64u;
  const uint64_t lowb = C128 ? (uint64_t)((t & 7u) * 16u) : (uint64_t)((t & 3u) * 16u);
  const int dthr = P.dnt - P.dtile;                              // diagonal terms with QL != 0
  const int dsm = dthr < kRegDiagSmem ? dthr : kRegDiagSmem;
  // raw amplitudes of the tile at `base`, 16-byte cp.async chunks into their
  // swizzled slots; base and the generator combinations have no bits below
  // bit 3, so the byte offset is (base ^ G) * kG | low bytes
  auto copy_tile = [&](uint64_t base) {
    const uint64_t baseb = base * kG;
#pragma unroll
    for (int i = 0; i < kNC; i++) {
      const uint64_t off = (baseb ^ gtab[gi0 + kGiStep * (uint32_t)i]) | lowb;
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                   :: "r"(sdst + kDstStep * (uint32_t)i), "l"(psi + off) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  double tot = 0.0;
  int kb = 0;
  for (uint64_t tix = blockIdx.x; tix < P.ntiles; tix += gridDim.x, kb ^= 1) {
    __syncthreads();                 // previous tile consumed; gtab and this tile's base written
    const uint64_t base = misc->base[kb];
    copy_tile(base);
    const bool next = tix + gridDim.x < P.ntiles;
    // While the copies are in flight, three warps stage this tile's signs in
    // parallel (each job's global loads are a dependent chain before the
    // barrier below): warp 0 the next tile's base and the QL = 0 diagonal sum,
    // warp 1 the pair groups' weights, warp 2 the other diagonal terms.
    const uint32_t lane = t & 31u, wid = t >> 5;
    if (wid == 0) {
      if (lane == 0 && next) misc->base[kb ^ 1] = tile_base(P, tix + gridDim.x);
      if (P.dtile > 0) {
        // sum of c_t (-1)^popc(base & Q_t) over the QL = 0 terms, float-float
        float kh = 0.f, kl = 0.f;
        for (int j = (int)lane; j < P.dtile; j += 32) {
          const TTerm* tt = &P.terms[P.dt0 + j];
          const uint32_t sb = (uint32_t)(__popcll(base & __ldg(&tt->q)) & 1) << 31;
          float s, e;
          two_sum(kh, __uint_as_float(__float_as_uint(__ldg(&tt->kh)) ^ sb), s, e);
          kh = s;
          kl = __fadd_rn(kl, __fadd_rn(e, __uint_as_float(__float_as_uint(__ldg(&tt->kl)) ^ sb)));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const float oh = __shfl_xor_sync(0xFFFFFFFFu, kh, o), ol = __shfl_xor_sync(0xFFFFFFFFu, kl, o);
          float s, e;
          two_sum(kh, oh, s, e);
          kh = s;
          kl = __fadd_rn(kl, __fadd_rn(ol, e));
        }
        if (lane == 0) { misc->kh = kh; misc->kl = kl; }
      }
    } else if (wid == 1) {
      // the staged pair groups' weights, signed by this tile's base
      for (int gi = (int)lane; gi < ngs; gi += 32) {
        const int t0 = __ldg(&P.groups[gi].t0), nt = __ldg(&P.groups[gi].nt);
        const uint32_t kind = __ldg(&P.groups[gi].kind);
        RegGW w;
        if (kind & 2u) {
          term_w2(&P.terms[t0], base, w.wh0, w.wl0);
          w.wh1 = w.wl1 = 0ull;
          if (nt > 1) term_w2(&P.terms[t0 + 1], base, w.wh1, w.wl1);
        } else {
          // the group's terms share FL, the weight (Re or Im w) and QL = 0: one summed weight
          float kh = 0.f, kl = 0.f;
          for (int k = 0; k < nt; k++) {
            const TTerm* tt = &P.terms[t0 + k];
            const uint32_t sb = (uint32_t)(__popcll(base & __ldg(&tt->q)) & 1) << 31;
            float s1, e1;
            two_sum(kh, __uint_as_float(__float_as_uint(__ldg(&tt->kh)) ^ sb), s1, e1);
            kh = s1;
            kl = __fadd_rn(kl, __fadd_rn(e1, __uint_as_float(__float_as_uint(__ldg(&tt->kl)) ^ sb)));
          }
          const uint32_t im = (kind & 1u) << 31;               // Im w: the second lane's weight negated
          w.wh0 = (uint64_t)__float_as_uint(kh) | ((uint64_t)(__float_as_uint(kh) ^ im) << 32);
          w.wl0 = (uint64_t)__float_as_uint(kl) | ((uint64_t)(__float_as_uint(kl) ^ im) << 32);
          w.wh1 = w.wl1 = 0ull;
        }
        sw[gi] = w;
      }
    } else if (wid == 2) {
      for (int j = (int)lane; j < dsm; j += 32) {
        const TTerm* tt = &P.terms[P.dt0 + P.dtile + j];
        const uint32_t sb = (uint32_t)(__popcll(base & __ldg(&tt->q)) & 1) << 31;
        RegDiag d;
        d.kh = __uint_as_float(__float_as_uint(__ldg(&tt->kh)) ^ sb);
        d.kl = __uint_as_float(__float_as_uint(__ldg(&tt->kl)) ^ sb);
        d.ql = __ldg(&tt->ql);
        d.pad = 0u;
        drec[j] = d;
      }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    uint64_t ah[16], al[16];
    uint64_t TH = 0ull, TL = 0ull;   // pair terms, packed float-float; the lanes are added per tile
    float th = 0.f, tl = 0.f;        // diagonal terms and the shared-memory groups
    // arrangement 0: raw -> split in registers, pair groups, diagonal terms, split form back
    reg_load<C128, true>(tile, 0, t, ah, al);
    const uint64_t sig0 = chain_sigma(reg_max(ah));
    if (P.garr[1] > P.garr[0]) reg_groups<C128>(P, sg, sw, P.garr[0], P.garr[1], 0, lb0, base, ah, al, sig0, zz, TH, TL);
    unsigned char* own = tile + reg_base<C128>(0, t);   // this thread's 16 amplitudes' chunks (arrangement 0)
    if (P.dnt > 0) {
      // |psi|^2 of the 16 amplitudes on the fixed grid of sigma: per lane
      // hi = fma(a, a, sigma) - sigma is exact, a multiple of ulp(sigma) =
      // 2^(E-23), and lo = the square's remainder (+ complex128's 2 hi*lo).
      // The lanes' hi add exactly, and so does every Walsh-Hadamard sum of
      // them (at most 32 mx^2 + 16 ulp <= 2^(E+1) = 2^24 ulp); lo adds in FP32.
      float wh[16], wl[16];
#pragma unroll
      for (int k = 0; k < 16; k++) {
        const uint64_t t1 = P2::fma2(ah[k], ah[k], sig0);
        const uint64_t r = P2::fma2(ah[k], ah[k], P2::sub2(sig0, t1));
        const uint64_t h2 = P2::sub2(t1, sig0);
        const uint64_t l2 = C128 ? P2::fma2(P2::add2(ah[k], ah[k]), al[k], r) : r;
        wh[k] = __fadd_rn(P2::lo32(h2), P2::hi32(h2));
        wl[k] = __fadd_rn(P2::lo32(l2), P2::hi32(l2));
      }
#pragma unroll
      for (int b = 1; b < 16; b <<= 1) {
#pragma unroll
        for (int k = 0; k < 16; k++) {
          if (!(k & b)) {
            const float xh = wh[k], yh = wh[k | b], xl = wl[k], yl = wl[k | b];
            wh[k] = __fadd_rn(xh, yh);
            wh[k | b] = __fsub_rn(xh, yh);
            wl[k] = __fadd_rn(xl, yl);
            wl[k | b] = __fsub_rn(xl, yl);
          }
        }
      }
      // QL = 0 terms: the tile-signed weight sum staged by warp 0, times W[0]
      if (P.dtile > 0) acc_scaled(th, tl, misc->kh, misc->kl, wh[0], wl[0]);
      if (dthr > 0) {
        // W[u] into this thread's own chunks, entry u at 8 (u ^ (lane & 15)) bytes:
        // the 16 lanes of a wavefront use 16 different bank pairs
        const uint32_t wsw = t & 15u;
#pragma unroll
        for (int k = 0; k < 16; k++) *(float2*)(own + 8 * ((uint32_t)k ^ wsw)) = make_float2(wh[k], wl[k]);
        // a term's sign at the thread's amplitudes: the tile's (in the staged
        // weight) times (-1)^popc(lb0 & QL); the register bits' part is in W[QL & 15]
        // two float-float accumulators on alternate terms: half the serial dependence
        float uh = 0.f, ul = 0.f;
        for (int j = 0; j < dsm; j++) {
          const RegDiag d = drec[j];
          const float2 w = *(const float2*)(own + 8 * ((d.ql & 15u) ^ wsw));
          const uint32_t sb = (uint32_t)(__popc(lb0 & d.ql) & 1) << 31;
          const float kh = __uint_as_float(__float_as_uint(d.kh) ^ sb), kl = __uint_as_float(__float_as_uint(d.kl) ^ sb);
          if (j & 1) acc_scaled(uh, ul, kh, kl, w.x, w.y);
          else acc_scaled(th, tl, kh, kl, w.x, w.y);
        }
        {
          float s1, e1;
          two_sum(th, uh, s1, e1);
          th = s1;
          tl = __fadd_rn(tl, __fadd_rn(ul, e1));
        }
        for (int j = dsm; j < dthr; j++) {
          const TTerm* tt = &P.terms[P.dt0 + P.dtile + j];
          const uint32_t ql = __ldg(&tt->ql);
          const float2 w = *(const float2*)(own + 8 * ((ql & 15u) ^ wsw));
          const uint32_t sb = (uint32_t)((__popcll(base & __ldg(&tt->q)) + __popc(lb0 & ql)) & 1) << 31;
          acc_scaled(th, tl, __uint_as_float(__float_as_uint(__ldg(&tt->kh)) ^ sb),
                     __uint_as_float(__float_as_uint(__ldg(&tt->kl)) ^ sb), w.x, w.y);
        }
      }
    }
    const bool later = P.garr[3] > P.garr[1] || P.ngroups > P.garr[3];
    if (later && (C128 || dthr > 0)) {
      // the split form (complex128) or the amplitudes themselves (complex64) back into the own chunks
      if constexpr (C128) {
#pragma unroll
        for (int r = 0; r < 16; r++)
          *(uint4*)(own + 16 * r) =
              make_uint4((uint32_t)ah[r], (uint32_t)(ah[r] >> 32), (uint32_t)al[r], (uint32_t)(al[r] >> 32));
      } else {
#pragma unroll
        for (int k = 0; k < 8; k++)
          *(uint4*)(own + 16 * k) =
              make_uint4((uint32_t)ah[2 * k], (uint32_t)(ah[2 * k] >> 32), (uint32_t)ah[2 * k + 1],
                         (uint32_t)(ah[2 * k + 1] >> 32));
      }
    }
    if (later) {
      __syncthreads();
      if (P.garr[2] > P.garr[1]) {
        reg_load<C128, false>(tile, 1, t, ah, al);
        reg_groups<C128>(P, sg, sw, P.garr[1], P.garr[2], 1, lb1, base, ah, al, chain_sigma(reg_max(ah)), zz, TH, TL);
      }
      if (P.garr[3] > P.garr[2]) {
        reg_load<C128, false>(tile, 2, t, ah, al);
        reg_groups<C128>(P, sg, sw, P.garr[2], P.garr[3], 2, lb2, base, ah, al, chain_sigma(reg_max(ah)), zz, TH, TL);
      }
      for (int gi = P.garr[3]; gi < P.ngroups; gi++) {
        TGroup g;
        g.fl = __ldg(&P.groups[gi].fl);
        g.pivot = __ldg(&P.groups[gi].pivot);
        g.t0 = __ldg(&P.groups[gi].t0);
        g.nt = __ldg(&P.groups[gi].nt);
        g.kind = __ldg(&P.groups[gi].kind);
        switch (g.kind) {
          case 0: tile_group<C128, false, false, true>(tile, P, g, base, zz, th, tl); break;
          case 1: tile_group<C128, true, false, true>(tile, P, g, base, zz, th, tl); break;
          case 2: tile_group<C128, false, true, true>(tile, P, g, base, zz, th, tl); break;
          default: tile_group<C128, true, true, true>(tile, P, g, base, zz, th, tl); break;
        }
      }
    }
    {
      // the tile's sum: both lanes of (TH, TL) and (th, tl), then two exact conversions
      float s, e, s2, e2;
      two_sum(P2::lo32(TH), P2::hi32(TH), s, e);
      two_sum(th, s, s2, e2);
      const float l = __fadd_rn(__fadd_rn(tl, e2), __fadd_rn(e, __fadd_rn(P2::lo32(TL), P2::hi32(TL))));
      tot += ArC128x::f2d(s2) + ArC128x::f2d(l);
    }
  }
  const double bs = block_sum(tot);
  if (threadIdx.x == 0) partial[blockIdx.x] = bs;
}

// ---- host planning --------------------------------------------------------
struct HTerm { uint64_t F, Q; int ny; double c; };

int parse_terms(int n, const qc_pauli_sum* H, std::vector<HTerm>& out) {
  if (!H || H->nterms < 0) return qc_fail(QC_ERR_ARG, "invalid Pauli sum");
  if (H->nterms > 0 && (!H->coeffs || !H->offsets)) return qc_fail(QC_ERR_ARG, "Pauli sum arrays are NULL");
  out.clear();
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
    out.push_back({F, Q, ny, H->coeffs[t]});
  }
  return QC_OK;
}

// GF(2) basis in reduced form: every vector has its own pivot (highest set
// bit) and no other vector has that bit set.
struct Basis {
  std::vector<uint64_t> v;
  // Reduce x by the basis; hc gets bit i for every vector i used.
  uint64_t reduce(uint64_t x, uint32_t* hc) const {
    uint32_t c = 0;
    for (size_t i = 0; i < v.size(); i++) {
      const int p = 63 - __builtin_clzll(v[i]);
      if ((x >> p) & 1ull) { x ^= v[i]; c |= 1u << i; }
    }
    if (hc) *hc = c;
    return x;
  }
  // Add a reduced, nonzero vector.
  void add(uint64_t r) {
    const int p = 63 - __builtin_clzll(r);
    for (auto& w : v)
      if ((w >> p) & 1ull) w ^= r;
    v.push_back(r);
  }
};

struct HPass {
  Basis basis;
  std::vector<uint64_t> flips;     // distinct flip masks assigned here
  double cost = 0.0;
};

struct TilePlan {
  std::vector<TPass> passes;       // term/group pointers filled in at upload
  std::vector<TTerm> terms;
  std::vector<TGroup> groups;
  std::vector<int> term_off, group_off;
};

double group_cost(uint64_t F, int nterms) {
  return F == 0 ? 4.0 + 0.08 * nterms : 1.0 + 0.3 * nterms;
}

int tile_plan(int n, bool c128, const std::vector<HTerm>& terms_in, TilePlan& plan) {
  // terms with the same flip and phase masks (hence the same nY) add up
  std::vector<HTerm> terms;
  {
    std::map<std::pair<uint64_t, uint64_t>, size_t> seen;
    for (const HTerm& t : terms_in) {
      auto it = seen.find({t.F, t.Q});
      if (it == seen.end()) {
        seen[{t.F, t.Q}] = terms.size();
        terms.push_back(t);
      } else {
        terms[it->second].c += t.c;
      }
    }
  }
  // n >= 12: the register-resident kernel, tiles of 2^12 amplitudes with 3 low
  // bits (runs of 8 amplitudes, 64 or 128 contiguous bytes) and 9 generators --
  // 3 passes for a nearest-neighbour chain of 30 qubits instead of 4 with 5
  // low bits and 7 generators
  const bool reg = n >= kRegL;
  const int Lmax = reg ? kRegL : (c128 ? 12 : 13), mdef = reg ? 3 : (c128 ? 5 : 6);
  const int L = std::min(n, Lmax);
  const int m = std::min(mdef, L);
  const int h = L - m;
  const uint64_t low = (1ull << m) - 1ull;
  // distinct flip masks, in order of first appearance
  std::vector<uint64_t> flips;
  std::map<uint64_t, int> count;
  for (const HTerm& t : terms) {
    if (!count.count(t.F)) flips.push_back(t.F);
    count[t.F]++;
  }
  std::vector<HPass> hp;
  // masks with bits above the low ones: first pass whose span holds them, or
  // that can still take one more generator
  for (uint64_t F : flips) {
    const uint64_t hi = F & ~low;
    if (!hi) continue;
    bool placed = false;
    for (HPass& p : hp) {
      const uint64_t r = p.basis.reduce(hi, nullptr);
      if (r == 0 || (int)p.basis.v.size() < h) {
        if (r) p.basis.add(r);
        p.flips.push_back(F);
        p.cost += group_cost(F, count[F]);
        placed = true;
        break;
      }
    }
    if (!placed) {
      hp.emplace_back();
      hp.back().basis.add(hi);
      hp.back().flips.push_back(F);
      hp.back().cost += group_cost(F, count[F]);
    }
  }
  if (hp.empty()) hp.emplace_back();
  // masks within the low bits (and the diagonal terms) fit every pass: cheapest
  for (uint64_t F : flips) {
    if (F & ~low) continue;
    HPass* best = &hp[0];
    for (HPass& p : hp)
      if (p.cost < best->cost) best = &p;
    best->flips.push_back(F);
    best->cost += group_cost(F, count[F]);
  }
  plan = TilePlan();
  for (HPass& p : hp) {
    // complete the basis with unit vectors at free bits above the low ones
    // (a unit vector at a non-pivot bit reduces to itself)
    for (int b = m; b < n && (int)p.basis.v.size() < h; b++) {
      const uint64_t r = p.basis.reduce(1ull << b, nullptr);
      if (r == (1ull << b)) p.basis.add(r);
    }
    if ((int)p.basis.v.size() != h) return qc_fail(QC_ERR_ARG, "internal: tile basis of rank %d, want %d",
                                                  (int)p.basis.v.size(), h);
    std::sort(p.basis.v.begin(), p.basis.v.end(),
              [](uint64_t a, uint64_t b) { return __builtin_clzll(a) > __builtin_clzll(b); });
    TPass P;
    std::memset(&P, 0, sizeof(P));
    P.ntiles = 1ull << (n - L);
    P.m = m;
    P.h = h;
    P.L = L;
    P.wb = L >= 8 ? 4 : 0;
    P.reg = reg ? 1 : 0;
    for (int i = 0; i < h; i++) {
      P.gen[i] = p.basis.v[i];
      P.piv[i] = 63 - __builtin_clzll(p.basis.v[i]);
    }
    const int t_begin = (int)plan.terms.size(), g_begin = (int)plan.groups.size();
    // local flip -> its terms (ordered for a deterministic layout)
    std::map<uint32_t, std::vector<const HTerm*>> by_fl;
    std::vector<const HTerm*> diag;
    auto local_q = [&](uint64_t Q) {
      uint32_t qh = 0;
      for (int i = 0; i < h; i++) qh |= (uint32_t)(__builtin_popcountll(P.gen[i] & Q) & 1) << i;
      return (qh << m) | (uint32_t)(Q & low);
    };
    std::vector<uint64_t> assigned(p.flips);
    std::sort(assigned.begin(), assigned.end());
    for (const HTerm& t : terms) {
      if (!std::binary_search(assigned.begin(), assigned.end(), t.F)) continue;
      if (t.F == 0) { diag.push_back(&t); continue; }
      uint32_t hc = 0;
      const uint64_t r = p.basis.reduce(t.F & ~low, &hc);
      if (r) return qc_fail(QC_ERR_ARG, "internal: flip mask outside the pass span");
      by_fl[(hc << m) | (uint32_t)(t.F & low)].push_back(&t);
    }
    static const double kw[4] = {2.0, -2.0, -2.0, 2.0};
    auto push_term = [&](const HTerm* t, bool pair) {
      TTerm x;
      const double k = pair ? t->c * kw[t->ny & 3] : t->c;
      x.q = t->Q;
      x.ql = local_q(t->Q);
      x.pad = 0u;
      x.kh = (float)k;
      x.kl = (float)(k - (double)x.kh);
      const bool im = pair && (t->ny & 1);
      x.kh2 = im ? -x.kh : x.kh;
      x.kl2 = im ? -x.kl : x.kl;
      plan.terms.push_back(x);
    };
    auto push_group = [&](uint32_t fl, uint32_t kind, const std::vector<const HTerm*>& v, size_t i0, size_t cnt) {
      TGroup g;
      g.fl = fl;
      g.pivot = 31 - __builtin_clz(fl);
      g.t0 = (int)plan.terms.size() - t_begin;
      g.nt = (int)cnt;
      g.kind = kind;
      for (size_t k = 0; k < cnt; k++) push_term(v[i0 + k], true);
      plan.groups.push_back(g);
    };
    // register-resident kernel: groups whose local flip mask lies in the local
    // bits [4a, 4a + 4) come first, arrangement a = 0, 1, 2; the rest read the
    // tile from shared memory
    auto arrangement = [&](uint32_t fl) {
      if (!reg) return 3;
      for (int a = 0; a < 3; a++)
        if ((fl & ~(15u << (4 * a))) == 0) return a;
      return 3;
    };
    P.qmask = 0;
    for (int a = 0; a < 4; a++) {
      P.garr[a] = (int)plan.groups.size() - g_begin;
      // an arrangement's Re-weighted unsigned groups of a single register bit
      // come first, in order of the bit (the kernel runs them without dispatch)
      auto single = [&](uint32_t fl) {
        const uint32_t r = a < 3 ? fl >> (4 * a) : 0u;
        return a < 3 && r != 0 && (r & (r - 1)) == 0;
      };
      for (int pass2 = 0; pass2 < 2; pass2++)
      for (auto& kv : by_fl) {
        if (arrangement(kv.first) != a) continue;
        // split by Re / Im weight and by whether the phase mask reaches into the tile
        std::vector<const HTerm*> part[4];
        for (const HTerm* t : kv.second) part[(t->ny & 1) | (local_q(t->Q) ? 2 : 0)].push_back(t);
        for (uint32_t kind = 0; kind < 4; kind++) {
          const std::vector<const HTerm*>& v = part[kind];
          if (v.empty()) continue;
          const bool quad = kind == 0 && single(kv.first);
          if (quad != (pass2 == 0)) continue;
          if (quad) P.qmask |= (int)((kv.first >> (4 * a)) << (4 * a));
          if (kind & 2u) {
            for (size_t i = 0; i < v.size(); i += kGroupTerms)
              push_group(kv.first, kind, v, i, std::min<size_t>(kGroupTerms, v.size() - i));
          } else {
            push_group(kv.first, kind, v, 0, v.size());
          }
        }
      }
    }
    // diagonal terms: those whose phase mask misses the tile's bits (QL = 0) first
    P.dt0 = (int)plan.terms.size() - t_begin;
    for (const HTerm* t : diag)
      if (local_q(t->Q) == 0) push_term(t, false);
    P.dtile = (int)plan.terms.size() - t_begin - P.dt0;
    for (const HTerm* t : diag)
      if (local_q(t->Q) != 0) push_term(t, false);
    P.dnt = (int)diag.size();
    P.ngroups = (int)plan.groups.size() - g_begin;
    plan.term_off.push_back(t_begin);
    plan.group_off.push_back(g_begin);
    plan.passes.push_back(P);
  }
  return QC_OK;
}

// Grow-only device buffer per device for the term and group tables.
std::map<int, std::pair<void*, size_t>> g_tables;

int get_tables(int device, size_t bytes, void** p) {
  auto& e = g_tables[device];
  if (e.second < bytes) {
    if (e.first) cudaFree(e.first);
    e.first = nullptr;
    e.second = 0;
    cudaError_t err = cudaMalloc(&e.first, bytes);
    if (err != cudaSuccess) { e.first = nullptr; return qc_cuda_fail(err, "cudaMalloc(term tables)"); }
    e.second = bytes;
  }
  *p = e.first;
  return QC_OK;
}

template <bool C128>
int launch_reg(const qc_state* s, const TPass& P, double* partial, int grid) {
  constexpr size_t kFixed = (size_t)reg_slots(C128) * 16 + ((size_t)8 << kRegH) + sizeof(RegMisc);
  if (P.m != kRegM || P.h != kRegH || P.L != kRegL)
    return qc_fail(QC_ERR_ARG, "internal: register-resident pass with m=%d h=%d L=%d", P.m, P.h, P.L);
  const int dthr = P.dnt - P.dtile;
  const int ngs = std::min(P.garr[3], kRegGroupSmem);
  const size_t smem = kFixed + (sizeof(RegGroup) + sizeof(RegGW)) * (size_t)ngs +
                      sizeof(RegDiag) * (size_t)std::min(dthr, kRegDiagSmem);
  static bool attr[64] = {false};
  const int dev = s->device;
  if (dev < 0 || dev >= 64 || !attr[dev]) {
    QC_CUDA(cudaFuncSetAttribute(k_pauli_reg<C128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(kFixed + (sizeof(RegGroup) + sizeof(RegGW)) * kRegGroupSmem +
                                       sizeof(RegDiag) * kRegDiagSmem)));
    QC_CUDA(cudaFuncSetAttribute(k_pauli_reg<C128>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared));
    if (dev >= 0 && dev < 64) attr[dev] = true;
  }
  k_pauli_reg<C128><<<grid, kTileThreads, smem, s->stream>>>((const unsigned char*)s->ptr, P, partial);
  QC_LAUNCHED("k_pauli_reg");
  return QC_OK;
}

template <bool C128>
int launch_tile(const qc_state* s, const TPass& P, double* partial, int grid) {
  const size_t smem = ((size_t)TileT<C128>::E << P.L) + ((size_t)8 << P.h);
  static bool attr[64] = {false};
  const int dev = s->device;
  if (dev >= 0 && dev < 64 && !attr[dev]) {
    QC_CUDA(cudaFuncSetAttribute(k_pauli_tile<C128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(((size_t)TileT<C128>::E << (C128 ? 12 : 13)) + (8 << kTileMaxH))));
    QC_CUDA(cudaFuncSetAttribute(k_pauli_tile<C128>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared));
    attr[dev] = true;
  }
  k_pauli_tile<C128><<<grid, kTileThreads, smem, s->stream>>>((const unsigned char*)s->ptr, P, partial);
  QC_LAUNCHED("k_pauli_tile");
  return QC_OK;
}

}  // namespace

extern "C" int qc_expect_passes(int n, int dtype, const qc_pauli_sum* H, int* npasses) {
  if (n < 1 || n > 36) return qc_fail(QC_ERR_ARG, "n=%d out of range 1..36", n);
  if (dtype != QC_C64 && dtype != QC_C128) return qc_fail(QC_ERR_ARG, "unknown dtype %d", dtype);
  if (!npasses) return qc_fail(QC_ERR_ARG, "npasses is NULL");
  std::vector<HTerm> terms;
  if (int rc = parse_terms(n, H, terms)) return rc;
  if (terms.empty()) { *npasses = 0; return QC_OK; }
  TilePlan plan;
  if (int rc = tile_plan(n, dtype == QC_C128, terms, plan)) return rc;
  *npasses = (int)plan.passes.size();
  return QC_OK;
}

extern "C" int qc_expect(const qc_state* s, const qc_pauli_sum* H, double* out) {
  if (int rc = qc_check_state(s)) return rc;
  if (!out) return qc_fail(QC_ERR_ARG, "out is NULL");
  std::vector<HTerm> terms;
  if (int rc = parse_terms(s->n, H, terms)) return rc;
  if (terms.empty()) { *out = 0.0; return QC_OK; }
  const bool c128 = s->dtype != QC_C64;
  TilePlan plan;
  if (int rc = tile_plan(s->n, c128, terms, plan)) return rc;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  std::vector<int> grids(plan.passes.size());
  size_t total = 0;
  for (size_t i = 0; i < plan.passes.size(); i++) {
    const int cap = qc_num_sms() * (plan.passes[i].reg ? reg_ctas_per_sm(c128) : 3);
    grids[i] = (int)std::min<uint64_t>(plan.passes[i].ntiles, (uint64_t)cap);
    total += grids[i];
  }
  void* scratch = nullptr;
  if (int rc = get_scratch(s->device, (total + 1) * sizeof(double), &scratch)) return rc;
  const size_t tbytes = plan.terms.size() * sizeof(TTerm);
  const size_t gbytes = std::max<size_t>(1, plan.groups.size()) * sizeof(TGroup);
  void* tables = nullptr;
  if (int rc = get_tables(s->device, tbytes + gbytes, &tables)) return rc;
  TTerm* dterms = (TTerm*)tables;
  TGroup* dgroups = (TGroup*)((char*)tables + tbytes);
  QC_CUDA(cudaMemcpyAsync(dterms, plan.terms.data(), tbytes, cudaMemcpyHostToDevice, s->stream));
  if (!plan.groups.empty())
    QC_CUDA(cudaMemcpyAsync(dgroups, plan.groups.data(), plan.groups.size() * sizeof(TGroup),
                            cudaMemcpyHostToDevice, s->stream));
  double* partial = (double*)scratch;
  size_t off = 0;
  for (size_t i = 0; i < plan.passes.size(); i++) {
    TPass P = plan.passes[i];
    P.terms = dterms + plan.term_off[i];
    P.groups = dgroups + plan.group_off[i];
    const int rc = P.reg ? (c128 ? launch_reg<true>(s, P, partial + off, grids[i])
                                 : launch_reg<false>(s, P, partial + off, grids[i]))
                         : (c128 ? launch_tile<true>(s, P, partial + off, grids[i])
                                 : launch_tile<false>(s, P, partial + off, grids[i]));
    if (rc) return rc;
    off += grids[i];
  }
  double result = 0.0;
  k_sum_partials<<<1, kThreads, 0, s->stream>>>(partial, (int)total, partial + total);
  QC_LAUNCHED("k_sum_partials");
  QC_CUDA(cudaMemcpyAsync(&result, partial + total, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  QC_CUDA(cudaStreamSynchronize(s->stream));
  *out = result;
  return qc_take_device_status("qc_expect");
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
  // Parse every term once (host memory only), then group the terms by flip
  // mask: a stable sort keeps each group in term order.  One sweep per group
  // and per kMaxTermsPerSweep terms of it.
  struct NaTerm { uint64_t F, Q; int ny, t; };
  std::vector<NaTerm> terms((size_t)H->nterms);
  for (int t = 0; t < H->nterms; t++) {
    NaTerm& x = terms[(size_t)t];
    x.t = t;
    if (int rc = na_term(s->n, H, t, &x.F, &x.Q, &x.ny)) return rc;
  }
  std::stable_sort(terms.begin(), terms.end(), [](const NaTerm& a, const NaTerm& b) { return a.F < b.F; });
  int nsweeps = 0;
  for (size_t a = 0; a < terms.size();) {
    size_t b = a;
    while (b < terms.size() && terms[b].F == terms[a].F) b++;
    nsweeps += (int)((b - a + kMaxTermsPerSweep - 1) / kMaxTermsPerSweep);
    a = b;
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
  for (size_t a = 0; a < terms.size();) {
    const uint64_t F = terms[a].F;
    size_t b = a;
    while (b < terms.size() && terms[b].F == F) b++;
    const uint64_t npairs = F ? N / 2 : N;
    const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((npairs + kThreads - 1) / kThreads, cap));
    for (size_t c = a; c < b; c += kMaxTermsPerSweep) {
      TermSet ts;
      std::memset(&ts, 0, sizeof(ts));
      ts.flip = F;
      ts.pivot = F ? 63 - __builtin_clzll(F) : -1;
      for (size_t u = c; u < b && ts.nterms < kMaxTermsPerSweep; u++) {
        ts.phase_mask[ts.nterms] = terms[u].Q;
        ts.coeff[ts.nterms] = H->coeffs[terms[u].t];
        ts.ipow[ts.nterms] = terms[u].ny & 3;
        ts.nterms++;
      }
      if (s->dtype == QC_C64)
        k_pauli_sweep<float2><<<grid, kThreads, 0, s->stream>>>((const float2*)s->ptr, npairs, ts, partial);
      else
        k_pauli_sweep<double2><<<grid, kThreads, 0, s->stream>>>((const double2*)s->ptr, npairs, ts, partial);
      k_sum_partials<<<1, kThreads, 0, s->stream>>>(partial, grid, sweep_sum + sw);
      QC_LAUNCHED("qc_expect_noalloc sweep");
      sw++;
    }
    a = b;
  }
  double result = 0.0;
  if (sw > 0) {
    k_sum_partials<<<1, kThreads, 0, s->stream>>>(sweep_sum, sw, final_sum);
    QC_LAUNCHED("qc_expect_noalloc final sum");
    QC_CUDA(cudaMemcpyAsync(&result, final_sum, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  }
  QC_CUDA(cudaStreamSynchronize(s->stream));
  *out = result;
  return qc_take_device_status("qc_expect_noalloc");
}
