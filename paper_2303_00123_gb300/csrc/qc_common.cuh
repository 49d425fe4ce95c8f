// qc_common.cuh -- shared definitions of the GB300 gate engine (device + host).
//
// Index convention (QCLAB++ Definition 1): qubit q of an n-qubit register is
// bit position p = n-1-q of the basis index, i.e. it has stride 2^p.  All
// kernels work with bit positions; the host converts qubit numbers once.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <cstring>

#include "qcgb300.h"

// --------------------------------------------------------------------------
// Library state handle
// --------------------------------------------------------------------------
struct qc_state {
  void* ptr;            // 2^n amplitudes, interleaved (re, im)
  int n;                // qubits
  int dtype;            // QC_C64 / QC_C128
  int owned;            // 1: allocated by qc_state_alloc
  int arith;            // qc_arith for QC_C128
  int device;           // CUDA device ordinal the memory lives on
  int fused_tc;         // 1: complex64 k-qubit blocks (k >= 3) on the tensor cores
  int packed;           // 1: float-float dense / phase sweeps use packed FP32 pairs
  long long wait_limit; // tensor-core MMA wait limit in polls (0: default; < 0: no poll)
  cudaStream_t stream;  // work queue
};

// --------------------------------------------------------------------------
// Errors (thread-local message, negative status codes)
// --------------------------------------------------------------------------
int qc_fail(int code, const char* fmt, ...);
int qc_cuda_fail(cudaError_t e, const char* what);
#define QC_CUDA(call)                                  \
  do {                                                 \
    cudaError_t qc_e_ = (call);                        \
    if (qc_e_ != cudaSuccess) return qc_cuda_fail(qc_e_, #call); \
  } while (0)
#define QC_LAUNCHED(what)                              \
  do {                                                 \
    cudaError_t qc_e_ = cudaGetLastError();            \
    if (qc_e_ != cudaSuccess) return qc_cuda_fail(qc_e_, what); \
  } while (0)

// Validate a handle; sets the CUDA device of the state current.
int qc_check_state(const qc_state* s);

// Validate target/control qubit numbers (range, distinctness, states 0/1).
int qc_check_qubits(int n, const int* t, int k, const int* c, const int* cs, int nc);

// Number of SMs of the current device (cached).
int qc_num_sms();

// --------------------------------------------------------------------------
// Index arithmetic
// --------------------------------------------------------------------------
// Insert a zero bit at position p of x (bits >= p move up by one).  Applying
// this for the sorted positions of the gate's targets and controls maps a
// loop counter j onto the first index of its group -- the paper's masks
// m_L, m_C, m_R of Alg. 1-3 (Eqs. (9)-(10), (16)-(19)), generalised to any
// number of positions as Sec. 2.4 describes.
__host__ __device__ __forceinline__ uint64_t qc_insert_zero(uint64_t x, int p) {
  const uint64_t lo = x & ((1ull << p) - 1ull);
  return ((x ^ lo) << 1) | lo;
}

#define QC_MAX_INS (QC_MAX_TARGETS + QC_MAX_CONTROLS)

// --------------------------------------------------------------------------
// 32-byte vector memory access (one DRAM sector per thread access)
// --------------------------------------------------------------------------
struct __align__(32) vec32 { uint32_t w[8]; };

__device__ __forceinline__ vec32 qc_ld32(const void* p) {
  vec32 v;
  asm volatile("ld.global.L1::no_allocate.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(v.w[0]), "=r"(v.w[1]), "=r"(v.w[2]), "=r"(v.w[3]),
                 "=r"(v.w[4]), "=r"(v.w[5]), "=r"(v.w[6]), "=r"(v.w[7])
               : "l"(p));
  return v;
}
__device__ __forceinline__ void qc_st32(void* p, const vec32& v) {
  asm volatile("st.global.v8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
               :: "l"(p), "r"(v.w[0]), "r"(v.w[1]), "r"(v.w[2]), "r"(v.w[3]),
                  "r"(v.w[4]), "r"(v.w[5]), "r"(v.w[6]), "r"(v.w[7])
               : "memory");
}

// --------------------------------------------------------------------------
// Arithmetic policies.  Each provides
//   V, E       -- amplitudes per 32-byte vector, bytes per amplitude
//   val_t      -- in-register amplitude
//   coef_t     -- in-kernel form of one complex matrix entry (make_coef on host)
//   load(v, e) / store(v, e, x) -- amplitude e of a 32-byte vector
//   dot<K>(row, x) = sum_k row[k] * x[k]
// Amplitudes a kernel does not change are never passed through load/store,
// so they stay bit-exact.
// --------------------------------------------------------------------------

// complex64 state, FP32 arithmetic.
struct ArC64 {
  static constexpr int V = 4;
  static constexpr int E = 8;
  struct val_t { float re, im; };
  struct coef_t { float re, im; };
  static __host__ coef_t make_coef(double re, double im) { return {(float)re, (float)im}; }
  using raw_t = float2;
  static __device__ __forceinline__ val_t from_raw(const raw_t& r) { return {r.x, r.y}; }
  static __device__ __forceinline__ raw_t to_raw(const val_t& x) { return make_float2(x.re, x.im); }
  static __device__ __forceinline__ val_t load(const vec32& v, int e) {
    return {__uint_as_float(v.w[2 * e]), __uint_as_float(v.w[2 * e + 1])};
  }
  static __device__ __forceinline__ void store(vec32& v, int e, const val_t& x) {
    v.w[2 * e] = __float_as_uint(x.re); v.w[2 * e + 1] = __float_as_uint(x.im);
  }
  template <int K>
  static __device__ __forceinline__ val_t dot(const coef_t* c, const val_t* x) {
    float re = 0.f, im = 0.f;
#pragma unroll
    for (int k = 0; k < K; k++) {
      re = fmaf(c[k].re, x[k].re, re); re = fmaf(-c[k].im, x[k].im, re);
      im = fmaf(c[k].re, x[k].im, im); im = fmaf(c[k].im, x[k].re, im);
    }
    return {re, im};
  }
};

// complex128 state, native FP64 arithmetic (bound by GB300's FP64 rate).
struct ArC128 {
  static constexpr int V = 2;
  static constexpr int E = 16;
  struct val_t { double re, im; };
  struct coef_t { double re, im; };
  static __host__ coef_t make_coef(double re, double im) { return {re, im}; }
  using raw_t = double2;
  static __device__ __forceinline__ val_t from_raw(const raw_t& r) { return {r.x, r.y}; }
  static __device__ __forceinline__ raw_t to_raw(const val_t& x) { return make_double2(x.re, x.im); }
  static __device__ __forceinline__ val_t load(const vec32& v, int e) {
    return {__hiloint2double((int)v.w[4 * e + 1], (int)v.w[4 * e]),
            __hiloint2double((int)v.w[4 * e + 3], (int)v.w[4 * e + 2])};
  }
  static __device__ __forceinline__ void store(vec32& v, int e, const val_t& x) {
    v.w[4 * e] = (uint32_t)__double2loint(x.re); v.w[4 * e + 1] = (uint32_t)__double2hiint(x.re);
    v.w[4 * e + 2] = (uint32_t)__double2loint(x.im); v.w[4 * e + 3] = (uint32_t)__double2hiint(x.im);
  }
  template <int K>
  static __device__ __forceinline__ val_t dot(const coef_t* c, const val_t* x) {
    double re = 0.0, im = 0.0;
#pragma unroll
    for (int k = 0; k < K; k++) {
      re = fma(c[k].re, x[k].re, re); re = fma(-c[k].im, x[k].im, re);
      im = fma(c[k].re, x[k].im, im); im = fma(c[k].im, x[k].re, im);
    }
    return {re, im};
  }
};

// complex128 state (IEEE binary64 in memory), float-float arithmetic on the
// FP32 and integer pipes.
//
// Why: GB300 executes FP64 FMA and f64<->f32 conversions at about 2 per clock
// per SM against 128 FP32 FMA, so a dense complex128 sweep done in FP64
// cannot keep up with HBM.  Here each input double is split exactly into two
// floats with integer bit operations (the double-single representation of
// Dekker 1971), products are formed error-free with an FMA (TwoProduct) and
// running sums with Knuth's TwoSum, and each real output is rebuilt from its
// two float parts (converted to doubles by integer bit operations) with a
// single FP64 add -- the only FP64-pipe instruction per output.
//
// Accuracy: the split keeps each input to 47 significant bits, rounded to
// nearest (relative error <= 2^-47, unbiased); each real output carries an
// error of about 2^-46 * sum_k |u_k| |x_k|.  Range: inputs with |x| < 2^-100 are flushed to
// zero (absolute error < 1e-30); |x| must stay below 2^127.
struct ArC128x {
  static constexpr int V = 2;
  static constexpr int E = 16;
  struct ff { float h, l; };
  struct val_t { ff re, im; };
  // One complex entry u = ur + i ui, split as ur = rh + rl, ui = ih + il.
  struct coef_t { float rh, rl, ih, il; };
  static __host__ coef_t make_coef(double re, double im) {
    coef_t c;
    c.rh = (float)re; c.rl = (float)(re - (double)c.rh);
    c.ih = (float)im; c.il = (float)(im - (double)c.ih);
    return c;
  }
  // IEEE double given as (low word, high word) -> (hi, lo) floats.
  static __device__ __forceinline__ ff split(uint32_t w0, uint32_t w1) {
    // hi: keep the sign, rebias the exponent (1023 -> 127) and keep the
    // leading 23 explicit mantissa bits (20 from w1, 3 from w0): truncation.
    const uint32_t t = w1 - 0x38000000u;
    uint32_t h = __funnelshift_l(w0, t, 3);
    h = (h & 0x7FFFFFFFu) | (w1 & 0x80000000u);
    // lo: the remaining 29 mantissa bits (w0 bits 28..0), rounded to the
    // nearest multiple of 2^6 units, i.e. m * 2^(E-46) with m <= 2^23; the
    // float difference (base + m) - base, with base = 2^(E-23), is exact and
    // equals that (an m of 2^23 carries into the exponent, still exact).
    // Rounding (not truncating) keeps the split unbiased: x is represented
    // to 47 significant bits, |x - (hi + lo)| <= 2^-47 |x|.
    const uint32_t base = (h & 0xFF800000u) - 0x0B800000u;
    const uint32_t m = ((w0 & 0x1FFFFFFFu) + 32u) >> 6;
    const float lo = __uint_as_float(base + m) - __uint_as_float(base);
    const bool tiny = (w1 & 0x7FFFFFFFu) < 0x39B00000u;  // |x| < 2^-100, or 0
    ff r;
    r.h = tiny ? 0.f : __uint_as_float(h);
    r.l = tiny ? 0.f : lo;
    return r;
  }
  // float -> IEEE double bits, exact for normal floats (zero/subnormal -> +-0).
  static __device__ __forceinline__ double f2d(float f) {
    const uint32_t b = __float_as_uint(f);
    const uint32_t m = b & 0x7FFFFFFFu;
    const bool z = m < 0x00800000u;
    const uint32_t hi = z ? (b & 0x80000000u) : (((m >> 3) + 0x38000000u) | (b & 0x80000000u));
    const uint32_t lo = z ? 0u : (b << 29);
    return __hiloint2double((int)hi, (int)lo);
  }
  static __device__ __forceinline__ val_t load(const vec32& v, int e) {
    return {split(v.w[4 * e], v.w[4 * e + 1]), split(v.w[4 * e + 2], v.w[4 * e + 3])};
  }
  using raw_t = double2;
  static __device__ __forceinline__ val_t from_raw(const raw_t& r) {
    return {split((uint32_t)__double2loint(r.x), (uint32_t)__double2hiint(r.x)),
            split((uint32_t)__double2loint(r.y), (uint32_t)__double2hiint(r.y))};
  }
  static __device__ __forceinline__ raw_t to_raw(const val_t& x) {
    return make_double2(f2d(x.re.h) + f2d(x.re.l), f2d(x.im.h) + f2d(x.im.l));
  }
  // x holds unnormalised (s, c) pairs; the double is s + c rounded once.
  static __device__ __forceinline__ void store(vec32& v, int e, const val_t& x) {
    const double re = f2d(x.re.h) + f2d(x.re.l);
    const double im = f2d(x.im.h) + f2d(x.im.l);
    v.w[4 * e] = (uint32_t)__double2loint(re); v.w[4 * e + 1] = (uint32_t)__double2hiint(re);
    v.w[4 * e + 2] = (uint32_t)__double2loint(im); v.w[4 * e + 3] = (uint32_t)__double2hiint(im);
  }
  // Running float-float accumulator: s is the rounded sum of the leading
  // products, c collects their exact rounding errors and the cross terms.
  struct acc_t { float s, c; };
  static __device__ __forceinline__ void acc_first(acc_t& a, float uh, float ul, const ff& x) {
    const float p = uh * x.h;
    a.s = p;
    a.c = fmaf(uh, x.h, -p);          // exact error of the product
    a.c = fmaf(uh, x.l, a.c);
    a.c = fmaf(ul, x.h, a.c);
  }
  static __device__ __forceinline__ void acc_add(acc_t& a, float uh, float ul, const ff& x) {
    const float p = uh * x.h;
    const float e = fmaf(uh, x.h, -p);
    const float t = a.s + p;          // TwoSum(s, p)
    const float z = t - a.s;
    const float err = (a.s - (t - z)) + (p - z);
    a.s = t;
    a.c += err + e;
    a.c = fmaf(uh, x.l, a.c);
    a.c = fmaf(ul, x.h, a.c);
  }
  template <int K>
  static __device__ __forceinline__ val_t dot(const coef_t* c, const val_t* x) {
    // re = sum ur*xr - ui*xi ;  im = sum ur*xi + ui*xr
    acc_t re, im;
    acc_first(re, c[0].rh, c[0].rl, x[0].re);
    acc_add(re, -c[0].ih, -c[0].il, x[0].im);
    acc_first(im, c[0].rh, c[0].rl, x[0].im);
    acc_add(im, c[0].ih, c[0].il, x[0].re);
#pragma unroll
    for (int k = 1; k < K; k++) {
      acc_add(re, c[k].rh, c[k].rl, x[k].re);
      acc_add(re, -c[k].ih, -c[k].il, x[k].im);
      acc_add(im, c[k].rh, c[k].rl, x[k].im);
      acc_add(im, c[k].ih, c[k].il, x[k].re);
    }
    val_t r;
    r.re.h = re.s; r.re.l = re.c;
    r.im.h = im.s; r.im.l = im.c;
    return r;
  }
};

// complex128 float-float arithmetic with packed FP32 pairs.  Same operations
// and order as ArC128x, but the real and imaginary accumulators travel
// together in one 64-bit register pair and every step is one .f32x2
// instruction (Blackwell executes add/mul/fma on FP32 pairs), which halves the
// issue slots of the arithmetic.  For a complex term u*x the pairs are
//   (Re, Im) += (ur, ur) * (xr, xi) + (-ui, ui) * (xi, xr).
struct ArC128p {
  static constexpr int V = 2;
  static constexpr int E = 16;
  using raw_t = double2;
  struct val_t { uint64_t h, l; };              // (re.h, im.h), (re.l, im.l)
  // per complex entry: pairs for the straight term (ur, ur) and the swapped
  // term (-ui, ui): hi, lo and the negated hi.
  struct coef_t { uint64_t ah, al, anh, bh, bl, bnh; };
  static __host__ __device__ uint64_t pk(float lo, float hi) {
    uint32_t a, b;
    memcpy(&a, &lo, 4);
    memcpy(&b, &hi, 4);
    return (uint64_t)a | ((uint64_t)b << 32);
  }
  static __host__ coef_t make_coef(double re, double im) {
    const float rh = (float)re, rl = (float)(re - (double)rh);
    const float ih = (float)im, il = (float)(im - (double)ih);
    coef_t c;
    c.ah = pk(rh, rh); c.al = pk(rl, rl); c.anh = pk(-rh, -rh);
    c.bh = pk(-ih, ih); c.bl = pk(-il, il); c.bnh = pk(ih, -ih);
    return c;
  }
  static __device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
    uint64_t d; asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b)); return d;
  }
  static __device__ __forceinline__ uint64_t sub2(uint64_t a, uint64_t b) {
    uint64_t d; asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b)); return d;
  }
  static __device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
    uint64_t d; asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b)); return d;
  }
  static __device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d; asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c)); return d;
  }
  static __device__ __forceinline__ uint64_t swp(uint64_t a) { return (a >> 32) | (a << 32); }
  static __device__ __forceinline__ val_t load(const vec32& v, int e) {
    const ArC128x::ff re = ArC128x::split(v.w[4 * e], v.w[4 * e + 1]);
    const ArC128x::ff im = ArC128x::split(v.w[4 * e + 2], v.w[4 * e + 3]);
    return {pk(re.h, im.h), pk(re.l, im.l)};
  }
  static __device__ __forceinline__ float lo32(uint64_t a) { return __uint_as_float((uint32_t)a); }
  static __device__ __forceinline__ float hi32(uint64_t a) { return __uint_as_float((uint32_t)(a >> 32)); }
  // x.h = (s_re, s_im), x.l = (c_re, c_im): the double is s + c rounded once.
  static __device__ __forceinline__ void store(vec32& v, int e, const val_t& x) {
    const double re = ArC128x::f2d(lo32(x.h)) + ArC128x::f2d(lo32(x.l));
    const double im = ArC128x::f2d(hi32(x.h)) + ArC128x::f2d(hi32(x.l));
    v.w[4 * e] = (uint32_t)__double2loint(re); v.w[4 * e + 1] = (uint32_t)__double2hiint(re);
    v.w[4 * e + 2] = (uint32_t)__double2loint(im); v.w[4 * e + 3] = (uint32_t)__double2hiint(im);
  }
  // s, c: running pair sums (see ArC128x::acc_add); en = p - u*x = -(product error)
  static __device__ __forceinline__ void first(uint64_t& s, uint64_t& c, uint64_t uh, uint64_t ul, uint64_t unh,
                                               uint64_t xh, uint64_t xl) {
    const uint64_t p = mul2(uh, xh);
    const uint64_t en = fma2(unh, xh, p);
    s = p;
    c = fma2(ul, xh, fma2(uh, xl, sub2(0ull, en)));
  }
  static __device__ __forceinline__ void add(uint64_t& s, uint64_t& c, uint64_t uh, uint64_t ul, uint64_t unh,
                                             uint64_t xh, uint64_t xl) {
    const uint64_t p = mul2(uh, xh);
    const uint64_t en = fma2(unh, xh, p);
    const uint64_t t = add2(s, p);
    const uint64_t z = sub2(t, s);
    const uint64_t err = add2(sub2(s, sub2(t, z)), sub2(p, z));
    s = t;
    c = add2(c, sub2(err, en));   // c + (err + e), the scalar form's association
    c = fma2(uh, xl, c);
    c = fma2(ul, xh, c);
  }
  template <int K>
  static __device__ __forceinline__ val_t dot(const coef_t* cf, const val_t* x) {
    uint64_t s, c;
    first(s, c, cf[0].ah, cf[0].al, cf[0].anh, x[0].h, x[0].l);
    add(s, c, cf[0].bh, cf[0].bl, cf[0].bnh, swp(x[0].h), swp(x[0].l));
#pragma unroll
    for (int k = 1; k < K; k++) {
      add(s, c, cf[k].ah, cf[k].al, cf[k].anh, x[k].h, x[k].l);
      add(s, c, cf[k].bh, cf[k].bl, cf[k].bnh, swp(x[k].h), swp(x[k].l));
    }
    return {s, c};
  }
};

// --------------------------------------------------------------------------
// Host-side gate description handed to the launchers
// --------------------------------------------------------------------------
enum qc_struct { QC_ST_DENSE = 0, QC_ST_PERM = 1, QC_ST_PHASE = 2 };

enum qc_op_kind { QC_OP_MATRIX = 0, QC_OP_LINEAR_PHASE = 1, QC_OP_PERMUTE = 2 };

struct qc_op {
  int kind;                     // qc_op_kind
  int k;                        // number of targets
  int tpos[QC_MAX_TARGETS];     // target bit positions, tpos[0] = MSB of U's index
  int nc;                       // controls
  int cpos[QC_MAX_CONTROLS];    // control bit positions
  int cval[QC_MAX_CONTROLS];    // control states
  double U[2 * 32 * 32];        // 2^k x 2^k complex, row-major (re, im)
  // QC_OP_LINEAR_PHASE: amplitudes whose `anchor` bit is 1 are multiplied by
  // exp(i (theta0 + sum_j bit_{lin_pos[j]} * lin_theta[j])) -- a run of
  // commuting (controlled) phase gates that all involve the anchor qubit.
  int anchor;
  int nlin;
  int lin_pos[QC_MAX_LIN];
  double lin_theta[QC_MAX_LIN];
  double theta0;
  // QC_OP_LINEAR_PHASE with pre = 1: the 2x2 matrix U on the anchor (k = 1,
  // tpos[0] = anchor) is applied first, in the same sweep.
  int pre;
  // QC_OP_PERMUTE: a run of SWAP gates on disjoint qubit pairs, i.e. the bit
  // positions perm_a[i] and perm_b[i] of every basis index trade values.
  int nperm;
  int perm_a[18], perm_b[18];
};

// Resolve a gate record (named or explicit matrix) into an op: validates the
// qubits, builds the matrix (host FP64) and converts qubits to bit positions.
int qc_gate_to_op(int n, const qc_gate& g, qc_op& op);

// Number of tensor-core tile waits that gave up on the current device and
// have not been reported yet (device counter; 0 normally).
int qc_tc_timeouts(int* count);
// For calls that have just synchronised their stream: QC_ERR_TIMEOUT (and the
// counter reset to 0) when a tensor-core wait on the current device gave up
// since the last report, else QC_OK.
int qc_take_device_status(const char* where);

// Launch plan of a circuit: one op per gate, or per fused block (fuse_k >= 2);
// with phase_runs, runs of commuting phase gates sharing a qubit become one
// QC_OP_LINEAR_PHASE op (taking along a 1-qubit op on the anchor just before
// the run) and runs of SWAPs on disjoint pairs one QC_OP_PERMUTE op.
#include <vector>
int qc_plan_ops(int n, const qc_gate* gates, int ngates, int fuse_k, std::vector<qc_op>& ops,
                bool phase_runs = false);

// Apply one (controlled) k-qubit gate given by its matrix; the launcher
// classifies the matrix (dense / permutation / diagonal) and picks a kernel.
int qc_launch_op(qc_state* s, const qc_op& op);
