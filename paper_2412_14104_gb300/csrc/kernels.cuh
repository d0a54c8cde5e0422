// Launch wrappers of the library's kernels (host-callable), grouped by file.
#pragma once

#include <algorithm>

#include "common.cuh"

namespace tatrg {

// Per-context counters of what was launched.
struct Stats {
  long launches = 0;
  long tc_launches = 0;
  double flops_f64 = 0.0;
  double flops_tc = 0.0;  // algorithmic flops routed to the tensor cores
  // optional device timing of the tensor-core kernels: pairs of events, reused
  bool timing = false;
  std::vector<cudaEvent_t> events;
  size_t used = 0;
  cudaEvent_t next_event() {
    if (used == events.size()) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) throw Error(TATRG_ECUDA, "cudaEventCreate failed");
      events.push_back(e);
    }
    return events[used++];
  }
  // sum of the recorded intervals (call after a synchronise); resets the pool
  double drain_ms() {
    double t = 0.0;
    for (size_t i = 0; i + 1 < used; i += 2) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, events[i], events[i + 1]) == cudaSuccess) t += ms;
    }
    used = 0;
    return t;
  }
  ~Stats() {
    for (auto e : events) cudaEventDestroy(e);
  }
};

// kernels_f64.cu ----------------------------------------------------------------------
// multiprocessors of the current device (cached per device ordinal)
int sm_count();
// raise a kernel's dynamic shared-memory limit to `bytes` on the current device (once)
void ensure_smem_attr(const void* fn, int bytes);
// raw Philox4x32-10 words of counter blocks first .. first + npairs - 1 (philox.cuh)
void philox_words(uint64_t seed, uint32_t sid, uint32_t replica, uint64_t first, int64_t npairs,
                  uint32_t* out, cudaStream_t s);
void gemm_f64(const GemmDesc& d, const double* A, const double* B, double* C, cudaStream_t s,
              Stats* st);
// Philox4x32-10 Gaussians; float_math evaluates Box-Muller in float (split-precision
// sketches), otherwise in double.  out must be 16-byte aligned with float_math.
void gaussian(uint64_t seed, uint32_t sid, uint32_t replica, int64_t n, double* out,
              cudaStream_t s, bool float_math = false);
// x viewed as [outer, n, inner] is multiplied along n by v^power (power 1, 2, -1, -2=rsqrt)
void scale_axis(double* x, const double* v, int64_t outer, int64_t n, int64_t inner, int power,
                cudaStream_t s);
// dst[off1(e)] = alpha * src[off0(e)] for e over the modes (s0: source, s1: destination)
void copy_modes(double* dst, const double* src, const ModeIdx& m, double alpha, cudaStream_t s);
void weighted_colsum(const double* X, int64_t F, int n, double* v, cudaStream_t s);
void flip_by_sign(double* X, int64_t F, int n, double* Y, int64_t G, const double* v,
                  cudaStream_t s);
// G (m x m) = X[:, a:a+m]^T W with the hashed basis weights W (F x m)
void multiplet_overlap(const double* X, int64_t F, int n, int a, int m, double* G, cudaStream_t s);
void trace_asb(const double* A, const double* sv, const double* B, int64_t F, int Da,
               double* out, cudaStream_t s);
void sum_all(const double* x, int64_t n, double* out, cudaStream_t s);
void ising_tensor(double beta, double h, int d, double* T, cudaStream_t s);
void fill(double* x, int64_t n, double v, cudaStream_t s);
void check_finite(const double* x, int64_t n, int* bad_dev, cudaStream_t s);

// linalg.cu ---------------------------------------------------------------------------
// largest n of the one-block Cholesky (its working matrix lives in shared memory)
int cholesky_max_n();
// Cholesky G = R^T R of an n x n SPD matrix (row-major); R upper (row-major, zero below).
// *status_dev = 0 on success, 1 when a pivot is not positive relative to its diagonal.
void cholesky(const double* G, int n, double* R, int* status_dev, double shift_rel,
              cudaStream_t s);
// inverse of an upper-triangular n x n matrix (row-major)
void tri_inverse(const double* R, int n, double* Rinv, cudaStream_t s);
// One-sided Jacobi SVD of a row-major m x n (m >= n): U (m x n), S (n), V (n x n) with
// S descending.  *status_dev = 0 converged, 1 not converged.
void jacobi_svd(const double* A, int64_t m, int n, double* U, double* S, double* V,
                int* status_dev, cudaStream_t s, Stats* st);
// The same SVD of a square matrix (32 <= n <= 160) through a column-pivoted QR of A^T and
// the Jacobi on R^T.
bool qrcp_svd_fits(int64_t m, int n);
void jacobi_svd_qrcp(const double* A, int64_t m, int n, double* U, double* S, double* V,
                     int* status_dev, cudaStream_t s, Stats* st);
// C (n x n) = A (n x n) * B (n x n), all row-major, small FP64 helper
void transpose(const double* A, int64_t rows, int64_t cols, double* At, cudaStream_t s);
// The same SVD with its workspace in a fixed file-scope device array (no allocation);
// synchronises the stream.
void jacobi_svd_noalloc(const double* A, int64_t m, int n, double* U, double* S, double* V,
                        cudaStream_t s);

// time limit of the cooperative Jacobi's grid-barrier waits on the current device
void set_barrier_limit_ns(unsigned long long ns);

// tc_gemm.cu --------------------------------------------------------------------------
// Split-precision tcgen05 GEMM on multi-mode operands: prec 1 = 3xTF32, 2 = BF16x3.
bool tc_available();
// reads (and optionally clears) the flag a timed-out tensor-core wait raises
int tc_error_flag(bool reset);
// two-CTA tile forms of the split-precision GEMM: 0 autotuned, 1 CTA pairs, 2 multicast
// clusters wherever they apply (M >= 1024), -1 never
void set_pair_mode(int mode);
// A Gaussian sketch operand that is generated while packing instead of read from memory
// (the element index is the operand offset the modes give).
struct GaussSrc {
  uint64_t seed = 0;
  uint32_t sid = 0, replica = 0;
};
// gen_b: B is that sketch (B must be null)
void gemm_tc(const GemmDesc& d, const double* A, const double* B, double* C, int prec,
             cudaStream_t s, Stats* st, const GaussSrc* gen_b = nullptr);
// The float64-grade contraction from exact tensor-core products of integer slices
// (TATRG_OZAKI).
void gemm_oz(const GemmDesc& d, const double* A, const double* B, double* C, cudaStream_t s,
             Stats* st);

}  // namespace tatrg
