// qc_state.cu -- state handles, errors, single-gate C entry points.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <new>

#include "qc_common.cuh"

namespace {
thread_local char g_err[512] = "";

// Qubit q of an n-qubit register is bit position n-1-q (Definition 1).
inline int bitpos(int n, int q) { return n - 1 - q; }

}  // namespace

int qc_check_qubits(int n, const int* t, int k, const int* c, const int* cs, int nc) {
  if (k < 1 || k > QC_MAX_TARGETS) return qc_fail(QC_ERR_ARG, "number of targets %d out of range 1..%d", k, QC_MAX_TARGETS);
  if (nc < 0 || nc > QC_MAX_CONTROLS) return qc_fail(QC_ERR_ARG, "number of controls %d out of range 0..%d", nc, QC_MAX_CONTROLS);
  if (nc > 0 && (c == nullptr || cs == nullptr)) return qc_fail(QC_ERR_ARG, "controls or control_states is NULL");
  int seen[64] = {0};
  for (int i = 0; i < k + nc; i++) {
    const int q = i < k ? t[i] : c[i - k];
    if (q < 0 || q >= n) return qc_fail(QC_ERR_ARG, "qubit %d out of range 0..%d", q, n - 1);
    if (seen[q]) return qc_fail(QC_ERR_ARG, "qubit %d used twice (targets and controls must be distinct)", q);
    seen[q] = 1;
    if (i >= k && cs[i - k] != 0 && cs[i - k] != 1)
      return qc_fail(QC_ERR_ARG, "control state %d is not 0 or 1", cs[i - k]);
  }
  return QC_OK;
}

namespace {
__global__ void k_set_basis_c64(float2* p, uint64_t x) { p[x] = make_float2(1.f, 0.f); }
__global__ void k_set_basis_c128(double2* p, uint64_t x) { p[x] = make_double2(1.0, 0.0); }
}  // namespace

int qc_fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

int qc_cuda_fail(cudaError_t e, const char* what) {
  return qc_fail(QC_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

int qc_num_sms() {
  static int sms[64] = {0};   // per device ordinal
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 132;
  if (dev >= 0 && dev < 64 && sms[dev] > 0) return sms[dev];
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) return 132;
  if (dev >= 0 && dev < 64) sms[dev] = v;
  return v;
}

int qc_check_state(const qc_state* s) {
  if (s == nullptr || s->ptr == nullptr) return qc_fail(QC_ERR_ARG, "state handle is NULL");
  int cur = -1;
  QC_CUDA(cudaGetDevice(&cur));
  if (cur != s->device) QC_CUDA(cudaSetDevice(s->device));
  return QC_OK;
}

extern "C" {

const char* qc_last_error(void) { return g_err; }
const char* qc_version(void) { return "qcgb300 0.1 (sm_103a)"; }

static size_t elem_size(int dtype) { return dtype == QC_C64 ? 8 : 16; }

static int new_handle(void* ptr, int n, int dtype, int owned, qc_state** out) {
  qc_state* s = new (std::nothrow) qc_state;
  if (!s) return qc_fail(QC_ERR_OOM, "host allocation failed");
  s->ptr = ptr;
  s->n = n;
  s->dtype = dtype;
  s->owned = owned;
  s->arith = QC_ARITH_AUTO;
  s->fused_tc = 1;
  s->packed = 2;
  s->wait_limit = 0;
  s->stream = nullptr;
  cudaGetDevice(&s->device);
  *out = s;
  return QC_OK;
}

int qc_state_alloc(int n, int dtype, qc_state** out) {
  if (!out) return qc_fail(QC_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n < 1 || n > 36) return qc_fail(QC_ERR_ARG, "n=%d out of range 1..36", n);
  if (dtype != QC_C64 && dtype != QC_C128) return qc_fail(QC_ERR_ARG, "unknown dtype %d", dtype);
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0) return qc_fail(QC_ERR_CUDA, "no CUDA device available");
  const size_t bytes = ((size_t)1 << n) * elem_size(dtype);
  void* p = nullptr;
  e = cudaMalloc(&p, bytes < 32 ? 32 : bytes);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return qc_fail(QC_ERR_OOM, "cudaMalloc of %zu bytes failed", bytes);
  }
  if (e != cudaSuccess) return qc_cuda_fail(e, "cudaMalloc");
  int rc = new_handle(p, n, dtype, 1, out);
  if (rc) { cudaFree(p); return rc; }
  rc = qc_state_set_basis(*out, 0);
  if (rc) { qc_state_free(*out); *out = nullptr; return rc; }
  QC_CUDA(cudaStreamSynchronize((*out)->stream));
  return QC_OK;
}

int qc_state_wrap(void* dev_ptr, int n, int dtype, qc_state** out) {
  if (!out) return qc_fail(QC_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!dev_ptr) return qc_fail(QC_ERR_ARG, "dev_ptr is NULL");
  if (n < 1 || n > 36) return qc_fail(QC_ERR_ARG, "n=%d out of range 1..36", n);
  if (dtype != QC_C64 && dtype != QC_C128) return qc_fail(QC_ERR_ARG, "unknown dtype %d", dtype);
  if (((uintptr_t)dev_ptr) % 32 != 0) return qc_fail(QC_ERR_ARG, "dev_ptr must be 32-byte aligned");
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, dev_ptr);
  if (e != cudaSuccess) return qc_cuda_fail(e, "cudaPointerGetAttributes");
  if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
    return qc_fail(QC_ERR_ARG, "dev_ptr is not device memory");
  int rc = new_handle(dev_ptr, n, dtype, 0, out);
  if (rc == QC_OK) (*out)->device = a.device;
  return rc;
}

int qc_state_free(qc_state* s) {
  if (!s) return QC_OK;
  int rc = QC_OK;
  if (s->owned && s->ptr) {
    cudaSetDevice(s->device);
    cudaError_t e = cudaFree(s->ptr);
    if (e != cudaSuccess) rc = qc_cuda_fail(e, "cudaFree");
  }
  delete s;
  return rc;
}

int qc_state_set_basis(qc_state* s, uint64_t x) {
  if (int rc = qc_check_state(s)) return rc;
  if (x >> s->n) return qc_fail(QC_ERR_ARG, "basis index out of range");
  const size_t bytes = ((size_t)1 << s->n) * elem_size(s->dtype);
  QC_CUDA(cudaMemsetAsync(s->ptr, 0, bytes, s->stream));
  if (s->dtype == QC_C64) k_set_basis_c64<<<1, 1, 0, s->stream>>>((float2*)s->ptr, x);
  else k_set_basis_c128<<<1, 1, 0, s->stream>>>((double2*)s->ptr, x);
  QC_LAUNCHED("set_basis");
  return QC_OK;
}

int qc_state_copy_to_host(const qc_state* s, void* host) {
  if (int rc = qc_check_state(s)) return rc;
  if (!host) return qc_fail(QC_ERR_ARG, "host is NULL");
  const size_t bytes = ((size_t)1 << s->n) * elem_size(s->dtype);
  QC_CUDA(cudaMemcpyAsync(host, s->ptr, bytes, cudaMemcpyDeviceToHost, s->stream));
  QC_CUDA(cudaStreamSynchronize(s->stream));
  return qc_take_device_status("qc_state_copy_to_host");
}

int qc_synchronize(const qc_state* s) {
  if (int rc = qc_check_state(s)) return rc;
  QC_CUDA(cudaStreamSynchronize(s->stream));
  return qc_take_device_status("qc_synchronize");
}

int qc_set_wait_limit(qc_state* s, long long polls) {
  if (!s) return qc_fail(QC_ERR_ARG, "state handle is NULL");
  s->wait_limit = polls;
  return QC_OK;
}

// Host -> device copy by the GPU's own 16-byte loads from page-locked host
// memory that CUDA has mapped into the device's address space.
__global__ void k_copy_from_mapped(uint4* __restrict__ dst, const uint4* __restrict__ src, size_t n16) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

int qc_state_copy_from_host(qc_state* s, const void* host) {
  if (int rc = qc_check_state(s)) return rc;
  if (!host) return qc_fail(QC_ERR_ARG, "host is NULL");
  const size_t bytes = ((size_t)1 << s->n) * elem_size(s->dtype);
  // Page-locked host memory mapped for the state's device (cudaHostRegister, cudaHostAlloc): a copy kernel
  // reading it (measured on GB300: 17 GB at 210 GB/s, where the copy engine gave
  // 58-66 GB/s for the same registered buffer); anything else: the copy engine.
  cudaPointerAttributes at;
  const cudaError_t ae = cudaPointerGetAttributes(&at, host);
  if (ae == cudaSuccess && at.type == cudaMemoryTypeHost && at.devicePointer && at.device == s->device &&
      ((uintptr_t)at.devicePointer % 16) == 0 && ((uintptr_t)s->ptr % 16) == 0 && bytes % 16 == 0) {
    k_copy_from_mapped<<<qc_num_sms() * 8, 512, 0, s->stream>>>((uint4*)s->ptr, (const uint4*)at.devicePointer,
                                                              bytes / 16);
    QC_LAUNCHED("k_copy_from_mapped");
    return QC_OK;
  }
  if (ae != cudaSuccess) cudaGetLastError();
  QC_CUDA(cudaMemcpyAsync(s->ptr, host, bytes, cudaMemcpyHostToDevice, s->stream));
  return QC_OK;
}

int qc_state_info(const qc_state* s, void** dev_ptr, int* n, int* dtype) {
  if (!s) return qc_fail(QC_ERR_ARG, "state handle is NULL");
  if (dev_ptr) *dev_ptr = s->ptr;
  if (n) *n = s->n;
  if (dtype) *dtype = s->dtype;
  return QC_OK;
}

int qc_set_stream(qc_state* s, void* stream) {
  if (!s) return qc_fail(QC_ERR_ARG, "state handle is NULL");
  s->stream = (cudaStream_t)stream;
  return QC_OK;
}

int qc_set_fused_tc(qc_state* s, int enable) {
  if (!s) return qc_fail(QC_ERR_ARG, "state handle is NULL");
  if (enable < 0 || enable > 4) return qc_fail(QC_ERR_ARG, "qc_set_fused_tc: enable must be 0 .. 4");
  s->fused_tc = enable;
  return QC_OK;
}

int qc_set_packed(qc_state* s, int enable) {
  if (!s) return qc_fail(QC_ERR_ARG, "state handle is NULL");
  if (enable < 0 || enable > 2) return qc_fail(QC_ERR_ARG, "qc_set_packed: enable must be 0, 1 or 2");
  s->packed = enable;
  return QC_OK;
}

int qc_device_status(int* tc_timeouts) {
  if (!tc_timeouts) return qc_fail(QC_ERR_ARG, "tc_timeouts is NULL");
  return qc_tc_timeouts(tc_timeouts);
}

int qc_set_arith(qc_state* s, int arith) {
  if (!s) return qc_fail(QC_ERR_ARG, "state handle is NULL");
  if (arith < QC_ARITH_AUTO || arith > QC_ARITH_F32X2) return qc_fail(QC_ERR_ARG, "unknown arith %d", arith);
  s->arith = arith;
  return QC_OK;
}

static int apply_generic(qc_state* s, const double* U, const int* targets, int k,
                         const int* controls, const int* cstates, int nc) {
  if (int rc = qc_check_state(s)) return rc;
  if (!U) return qc_fail(QC_ERR_ARG, "matrix is NULL");
  if (!targets) return qc_fail(QC_ERR_ARG, "targets is NULL");
  if (int rc = qc_check_qubits(s->n, targets, k, controls, cstates, nc)) return rc;
  qc_op op;
  op.kind = QC_OP_MATRIX;
  op.k = k;
  for (int i = 0; i < k; i++) op.tpos[i] = bitpos(s->n, targets[i]);
  op.nc = nc;
  for (int i = 0; i < nc; i++) { op.cpos[i] = bitpos(s->n, controls[i]); op.cval[i] = cstates[i]; }
  std::memcpy(op.U, U, sizeof(double) * 2 * (size_t)(1 << k) * (1 << k));
  return qc_launch_op(s, op);
}

int qc_apply_1q(qc_state* s, const double U[8], int target) {
  return apply_generic(s, U, &target, 1, nullptr, nullptr, 0);
}

int qc_apply_c1q(qc_state* s, const double U[8], const int* controls, const int* control_states,
                 int ncontrols, int target) {
  return apply_generic(s, U, &target, 1, controls, control_states, ncontrols);
}

int qc_apply_2q(qc_state* s, const double U4[32], int q0, int q1) {
  const int t[2] = {q0, q1};
  return apply_generic(s, U4, t, 2, nullptr, nullptr, 0);
}

int qc_apply_kq(qc_state* s, const double* U, const int* qubits, int k, const int* controls,
                const int* control_states, int ncontrols) {
  return apply_generic(s, U, qubits, k, controls, control_states, ncontrols);
}

}  // extern "C"
