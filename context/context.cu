// Context measurements beside the subdomain-ILU0 path (not part of it):
//
//  * the vendor baseline: cuSPARSE global block ILU0 (bsrilu02, one
//    factorisation of the whole matrix, no decomposition), its two triangular
//    solves (bsrsv2, lower with unit diagonal, then upper) as the
//    preconditioner apply, and the vendor BSR SpMV (bsrmv), on the same matrix
//    and GPU as the library's path; this is the "global ILU0" the paper's
//    decomposition replaces (Section 3.2 drops the inter-subdomain blocks so
//    the solves need no cross-block synchronisation);
//  * the FP64 FMA issue rate of the GPU, which bounds the FP64 apply
//    alongside HBM bandwidth (an FP64 3x3 block costs 9 FMAs per 72 bytes).
//
// Plain C ABI; device buffers are allocated here with cudaMalloc (this is a
// measurement harness, not the allocation-free library). Every entry point
// returns 0 on success, 1 for a CUDA error, 2 for a cuSPARSE error, 3 for a
// zero pivot in bsrilu02 and 4 for invalid arguments.
#include <cuda_runtime.h>
#include <cusparse.h>

#include <cstdint>
#include <cstring>

namespace {

struct VendorIlu0 {
  cusparseHandle_t h = nullptr;
  cusparseMatDescr_t dM = nullptr, dL = nullptr, dU = nullptr;
  bsrilu02Info_t iM = nullptr;
  bsrsv2Info_t iL = nullptr, iU = nullptr;
  int mb = 0, nnzb = 0;
  int* row_ptr = nullptr;
  int* col = nullptr;
  double* lu = nullptr;   // factors (in place of A)
  double* a = nullptr;    // A itself, for the SpMV
  double* tmp = nullptr;  // L solve output
  void* buf = nullptr;
};

constexpr cusparseDirection_t kDir = CUSPARSE_DIRECTION_ROW;  // 3x3 blocks stored row-major
constexpr cusparseSolvePolicy_t kPolicy = CUSPARSE_SOLVE_POLICY_USE_LEVEL;
constexpr int kBlockDim = 3;

int free_all(VendorIlu0* v) {
  if (!v) return 0;
  if (v->iM) cusparseDestroyBsrilu02Info(v->iM);
  if (v->iL) cusparseDestroyBsrsv2Info(v->iL);
  if (v->iU) cusparseDestroyBsrsv2Info(v->iU);
  if (v->dM) cusparseDestroyMatDescr(v->dM);
  if (v->dL) cusparseDestroyMatDescr(v->dL);
  if (v->dU) cusparseDestroyMatDescr(v->dU);
  if (v->h) cusparseDestroy(v->h);
  cudaFree(v->row_ptr);
  cudaFree(v->col);
  cudaFree(v->lu);
  cudaFree(v->a);
  cudaFree(v->tmp);
  cudaFree(v->buf);
  delete v;
  return 0;
}

__global__ void fma_chains(double* out, int iters, double a, double b) {
  double x0 = threadIdx.x * 1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  double x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

}  // namespace

#define CU(x)                              \
  do {                                     \
    if ((x) != cudaSuccess) {              \
      free_all(v);                         \
      return 1;                            \
    }                                      \
  } while (0)
#define SP(x)                                   \
  do {                                          \
    if ((x) != CUSPARSE_STATUS_SUCCESS) {       \
      free_all(v);                              \
      return 2;                                 \
    }                                           \
  } while (0)

extern "C" {

// Global block ILU0 of A (host BSR arrays, 3x3 row-major blocks, sorted
// columns, diagonal present): copies A to the device, runs the analyses and
// the factorisation, and reports their wall time in *setup_ms.
int ctx_vendor_ilu0_create(int32_t mb, int64_t nnzb, const int32_t* row_ptr, const int32_t* col, const double* val,
                           void** out, double* setup_ms) {
  if (!out || !row_ptr || !col || !val || mb <= 0 || nnzb <= 0 || nnzb > INT32_MAX) return 4;
  VendorIlu0* v = new VendorIlu0;
  v->mb = mb;
  v->nnzb = (int)nnzb;
  const size_t vb = sizeof(double) * 9 * (size_t)nnzb;
  CU(cudaMalloc(&v->row_ptr, sizeof(int) * (mb + 1)));
  CU(cudaMalloc(&v->col, sizeof(int) * nnzb));
  CU(cudaMalloc(&v->lu, vb));
  CU(cudaMalloc(&v->a, vb));
  CU(cudaMalloc(&v->tmp, sizeof(double) * 3 * (size_t)mb));
  CU(cudaMemcpy(v->row_ptr, row_ptr, sizeof(int) * (mb + 1), cudaMemcpyHostToDevice));
  CU(cudaMemcpy(v->col, col, sizeof(int) * nnzb, cudaMemcpyHostToDevice));
  CU(cudaMemcpy(v->a, val, vb, cudaMemcpyHostToDevice));
  CU(cudaMemcpy(v->lu, v->a, vb, cudaMemcpyDeviceToDevice));
  SP(cusparseCreate(&v->h));
  SP(cusparseCreateMatDescr(&v->dM));
  SP(cusparseSetMatIndexBase(v->dM, CUSPARSE_INDEX_BASE_ZERO));
  SP(cusparseSetMatType(v->dM, CUSPARSE_MATRIX_TYPE_GENERAL));
  SP(cusparseCreateMatDescr(&v->dL));
  SP(cusparseSetMatIndexBase(v->dL, CUSPARSE_INDEX_BASE_ZERO));
  SP(cusparseSetMatType(v->dL, CUSPARSE_MATRIX_TYPE_GENERAL));
  SP(cusparseSetMatFillMode(v->dL, CUSPARSE_FILL_MODE_LOWER));
  SP(cusparseSetMatDiagType(v->dL, CUSPARSE_DIAG_TYPE_UNIT));
  SP(cusparseCreateMatDescr(&v->dU));
  SP(cusparseSetMatIndexBase(v->dU, CUSPARSE_INDEX_BASE_ZERO));
  SP(cusparseSetMatType(v->dU, CUSPARSE_MATRIX_TYPE_GENERAL));
  SP(cusparseSetMatFillMode(v->dU, CUSPARSE_FILL_MODE_UPPER));
  SP(cusparseSetMatDiagType(v->dU, CUSPARSE_DIAG_TYPE_NON_UNIT));
  SP(cusparseCreateBsrilu02Info(&v->iM));
  SP(cusparseCreateBsrsv2Info(&v->iL));
  SP(cusparseCreateBsrsv2Info(&v->iU));
  const cusparseOperation_t nt = CUSPARSE_OPERATION_NON_TRANSPOSE;
  int sM = 0, sL = 0, sU = 0;
  SP(cusparseDbsrilu02_bufferSize(v->h, kDir, mb, v->nnzb, v->dM, v->lu, v->row_ptr, v->col, kBlockDim, v->iM, &sM));
  SP(cusparseDbsrsv2_bufferSize(v->h, kDir, nt, mb, v->nnzb, v->dL, v->lu, v->row_ptr, v->col, kBlockDim, v->iL,
                                &sL));
  SP(cusparseDbsrsv2_bufferSize(v->h, kDir, nt, mb, v->nnzb, v->dU, v->lu, v->row_ptr, v->col, kBlockDim, v->iU,
                                &sU));
  int sb = sM > sL ? sM : sL;
  sb = sb > sU ? sb : sU;
  CU(cudaMalloc(&v->buf, (size_t)sb));
  CU(cudaDeviceSynchronize());
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  CU(cudaEventRecord(e0));
  SP(cusparseDbsrilu02_analysis(v->h, kDir, mb, v->nnzb, v->dM, v->lu, v->row_ptr, v->col, kBlockDim, v->iM,
                                kPolicy, v->buf));
  int pos = -1;
  if (cusparseXbsrilu02_zeroPivot(v->h, v->iM, &pos) == CUSPARSE_STATUS_ZERO_PIVOT) {
    free_all(v);
    return 3;
  }
  SP(cusparseDbsrsv2_analysis(v->h, kDir, nt, mb, v->nnzb, v->dL, v->lu, v->row_ptr, v->col, kBlockDim, v->iL,
                              kPolicy, v->buf));
  SP(cusparseDbsrsv2_analysis(v->h, kDir, nt, mb, v->nnzb, v->dU, v->lu, v->row_ptr, v->col, kBlockDim, v->iU,
                              kPolicy, v->buf));
  SP(cusparseDbsrilu02(v->h, kDir, mb, v->nnzb, v->dM, v->lu, v->row_ptr, v->col, kBlockDim, v->iM, kPolicy,
                       v->buf));
  CU(cudaEventRecord(e1));
  CU(cudaEventSynchronize(e1));
  if (cusparseXbsrilu02_zeroPivot(v->h, v->iM, &pos) == CUSPARSE_STATUS_ZERO_PIVOT) {
    free_all(v);
    return 3;
  }
  float ms = 0.f;
  CU(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (setup_ms) *setup_ms = ms;
  *out = v;
  return 0;
}

// z = U^-1 L^-1 r (device vectors of 3*mb doubles, natural order) on `stream`.
int ctx_vendor_ilu0_apply(void* h, const double* r, double* z, void* stream) {
  VendorIlu0* v = static_cast<VendorIlu0*>(h);
  if (!v || !r || !z) return 4;
  const double one = 1.0;
  const cusparseOperation_t nt = CUSPARSE_OPERATION_NON_TRANSPOSE;
  if (cusparseSetStream(v->h, (cudaStream_t)stream) != CUSPARSE_STATUS_SUCCESS) return 2;
  if (cusparseDbsrsv2_solve(v->h, kDir, nt, v->mb, v->nnzb, &one, v->dL, v->lu, v->row_ptr, v->col, kBlockDim, v->iL,
                            r, v->tmp, kPolicy, v->buf) != CUSPARSE_STATUS_SUCCESS)
    return 2;
  if (cusparseDbsrsv2_solve(v->h, kDir, nt, v->mb, v->nnzb, &one, v->dU, v->lu, v->row_ptr, v->col, kBlockDim, v->iU,
                            v->tmp, z, kPolicy, v->buf) != CUSPARSE_STATUS_SUCCESS)
    return 2;
  return 0;
}

// y = A x with the vendor BSR SpMV.
int ctx_vendor_spmv(void* h, const double* x, double* y, void* stream) {
  VendorIlu0* v = static_cast<VendorIlu0*>(h);
  if (!v || !x || !y) return 4;
  const double one = 1.0, zero = 0.0;
  if (cusparseSetStream(v->h, (cudaStream_t)stream) != CUSPARSE_STATUS_SUCCESS) return 2;
  if (cusparseDbsrmv(v->h, kDir, CUSPARSE_OPERATION_NON_TRANSPOSE, v->mb, v->mb, v->nnzb, &one, v->dM, v->a,
                     v->row_ptr, v->col, kBlockDim, x, &zero, y) != CUSPARSE_STATUS_SUCCESS)
    return 2;
  return 0;
}

// Copy the factors (L strictly below, U on and above the diagonal blocks, in
// A's pattern) to host memory of 9*nnzb doubles.
int ctx_vendor_ilu0_factors(void* h, double* host) {
  VendorIlu0* v = static_cast<VendorIlu0*>(h);
  if (!v || !host) return 4;
  return cudaMemcpy(host, v->lu, sizeof(double) * 9 * (size_t)v->nnzb, cudaMemcpyDeviceToHost) == cudaSuccess ? 0 : 1;
}

int ctx_vendor_ilu0_destroy(void* h) { return free_all(static_cast<VendorIlu0*>(h)); }

// FP64 FMA rate of the current device: 8 independent FMA chains per thread,
// 8 blocks of 256 threads per SM; the second of two launches is timed.
// *gflops receives FP64 GFLOP/s (2 flops per FMA).
int ctx_fp64_fma_rate(int iters, double* gflops) {
  if (!gflops || iters <= 0) return 4;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  const int blocks = sms * 8, threads = 256;
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double) * blocks * threads) != cudaSuccess) return 1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float ms = 0.f;
  for (int rep = 0; rep < 2; ++rep) {
    cudaEventRecord(e0);
    fma_chains<<<blocks, threads>>>(out, iters, 0.999, 1e-3);
    cudaEventRecord(e1);
  }
  cudaError_t e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess || ms <= 0.f) return 1;
  *gflops = 2.0 * 8 * (double)iters * blocks * threads / (ms * 1e-3) / 1e9;
  return 0;
}

}  // extern "C"
