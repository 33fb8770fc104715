// cimmino_aat_noalloc: C = A A^T into caller device buffers without any device
// allocation.  Some callers cannot let a library allocate device memory: an embedder
// whose device memory is reserved by its own caching allocator or capped by a fixed
// budget, or a latency-bound loop that cannot afford cudaMalloc / cudaFree (which may
// block the host and synchronise the device).  They can still build the row
// inner-product graph here.  The working arrays of the SpGEMM (transpose of A, row
// counts, scan partials, overflow list) live in one file-scope device array of a fixed
// size, which every GPU that loads this library holds until the process exits.  The call
// is host-synchronous: it reads counts back between its stages.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>

#include "internal.cuh"

using namespace cimmino;

namespace {

// Size limits of the static scratch: n <= 262,144 rows, nnz(A) <= 2,097,152.
constexpr int64_t kNaRows = int64_t(1) << 18;
constexpr int64_t kNaNnz = int64_t(1) << 21;

constexpr size_t al256(size_t b) { return (b + 255) & ~size_t(255); }
constexpr size_t kScanTmp = kNaRows / 2048 + 2;  // chunk totals of the 3-pass scan
// byte offsets of the pieces of the scratch array
constexpr size_t kOffCp = 0;                                           // int64 [n+1]
constexpr size_t kOffWork = kOffCp + al256(8 * (kNaRows + 1));         // int64 [2n]
constexpr size_t kOffCnt = kOffWork + al256(16 * kNaRows);             // int64 [n]
constexpr size_t kOffTmp = kOffCnt + al256(8 * kNaRows);               // int64 [kScanTmp]
constexpr size_t kOffOvf = kOffTmp + al256(8 * kScanTmp);              // int32 [n+1]
constexpr size_t kOffFlag = kOffOvf + al256(4 * (kNaRows + 1));        // int32 [4]
constexpr size_t kOffRi = kOffFlag + 256;                              // int32 [nnz]
constexpr size_t kOffCv = kOffRi + al256(4 * kNaNnz);                  // double [nnz]
constexpr size_t kScratchBytes = kOffCv + al256(8 * kNaNnz);           // ~33 MB

}  // namespace

static __device__ __align__(256) unsigned char g_aat_scratch[kScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
unsigned char *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  The host-side symbol
// is only a stand-in, so the address is looked up once per device (with that device
// current) and cached for the life of the process; a cudaDeviceReset() would reload the
// module at a possibly different address, so the entry point is documented as unusable
// on a device after a reset.
unsigned char *scratch_on_current_device() {
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) fail(CIMMINO_EUNSUPPORTED, "device index out of range");
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_aat_scratch);
    if (e != cudaSuccess || p == nullptr)
      fail(CIMMINO_ECUDA, std::string("cudaGetSymbolAddress of the scratch array failed: ") +
                              cudaGetErrorString(e));
    g_scratch_addr[dev] = static_cast<unsigned char *>(p);
  }
  return g_scratch_addr[dev];
}

}  // namespace

extern "C" {

int cimmino_aat_noalloc(const cimmino_csr *A, void *stream, int64_t *nnz, int64_t *row_ptr,
                        int32_t *col_idx, double *val, int64_t capacity) {
  if (!A || !nnz || !row_ptr) {
    record_last_error("invalid argument (NULL A, nnz or row_ptr)");
    return CIMMINO_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  try {
    const int64_t N = A->n, NNZ = A->nnz;
    if (!A->on_device) fail(CIMMINO_EINVAL, "A must be in device memory (on_device = 1)");
    if (N <= 0 || NNZ < 0 || !A->row_ptr || !A->col_idx || (NNZ > 0 && !A->val))
      fail(CIMMINO_EINVAL, "bad CSR header");
    if (N > kNaRows || NNZ > kNaNnz)
      fail(CIMMINO_EUNSUPPORTED, "cimmino_aat_noalloc supports n <= 262144 and nnz <= 2097152");
    unsigned char *base = scratch_on_current_device();
    int64_t *cp = reinterpret_cast<int64_t *>(base + kOffCp);
    int64_t *work = reinterpret_cast<int64_t *>(base + kOffWork);
    int64_t *cnt = reinterpret_cast<int64_t *>(base + kOffCnt);
    int64_t *tmp = reinterpret_cast<int64_t *>(base + kOffTmp);
    int32_t *ovf = reinterpret_cast<int32_t *>(base + kOffOvf);
    int32_t *flag = reinterpret_cast<int32_t *>(base + kOffFlag);
    int32_t *ri = reinterpret_cast<int32_t *>(base + kOffRi);
    double *cv = reinterpret_cast<double *>(base + kOffCv);
    // the array keeps the previous call's contents: clear what must start at zero
    CUDA_TRY(cudaMemsetAsync(flag, 0, 4 * sizeof(int32_t), s));
    launch_validate_csr(A->row_ptr, A->col_idx, N, NNZ, flag, s);
    int32_t hf = 0;
    CUDA_TRY(cudaMemcpyAsync(&hf, flag, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (hf) fail(CIMMINO_EINVAL, "malformed CSR");
    const int64_t tl = scan_tmp_len(N);
    launch_transpose(A->row_ptr, A->col_idx, A->val, N, NNZ, cp, ri, cv, work, tmp, tl, s);
    spgemm_count(A->row_ptr, A->col_idx, cp, ri, N, cnt, ovf + 1, ovf, s);
    int32_t novf = 0;
    CUDA_TRY(cudaMemcpyAsync(&novf, ovf, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (novf > 0) {
      spgemm_overflow(A->row_ptr, A->col_idx, A->val, cp, ri, ovf + 1, novf, cnt, nullptr, nullptr,
                      nullptr, flag + 1, s);
      CUDA_TRY(cudaMemcpyAsync(&hf, flag + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      CUDA_TRY(cudaStreamSynchronize(s));
      if (hf) fail(CIMMINO_EUNSUPPORTED, "a row of A A^T has more than 8192 structural candidates");
    }
    launch_scan_counts(cnt, row_ptr, N, tmp, tl, s);
    int64_t nc = 0;
    CUDA_TRY(cudaMemcpyAsync(&nc, row_ptr + N, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    *nnz = nc;
    if (col_idx && val) {
      if (capacity < nc)
        fail(CIMMINO_EINVAL, "capacity " + std::to_string(capacity) + " < nnz(C) = " +
                                 std::to_string(nc));
      spgemm_fill(A->row_ptr, A->col_idx, A->val, cp, ri, cv, N, row_ptr, col_idx, val, s);
      if (novf > 0)
        spgemm_overflow(A->row_ptr, A->col_idx, A->val, cp, ri, ovf + 1, novf, cnt, row_ptr,
                        col_idx, val, flag + 1, s);
    }
    CUDA_TRY(cudaStreamSynchronize(s));
    CUDA_TRY(cudaGetLastError());
    return CIMMINO_OK;
  } catch (const Error &e) {
    record_last_error(e.msg);
    return e.code;
  }
}

}  // extern "C"
