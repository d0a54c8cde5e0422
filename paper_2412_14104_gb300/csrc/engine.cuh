// Host-side building blocks of the RG step: contraction dispatch, orthonormalisation,
// small SVDs and the randomized SVDs (Halko, Martinsson & Tropp 2011, Alg. 4.4 + 5.1).
#pragma once

#include <functional>

#include "kernels.cuh"

namespace tatrg {

// A device matrix, row-major rows x cols.
struct DMat {
  DevBuf buf;
  int64_t rows = 0, cols = 0;
  double* p() const { return buf.d(); }
};

struct OrthResult {
  DMat Q;  // m x k
  DMat R;  // k x n (upper triangular when k == n)
  int k = 0;
};

struct SvdResult {
  DMat U;  // m x r
  DMat V;  // n x r
  DevBuf S;
  std::vector<double> s;  // host copy, descending
  int r = 0;
};

class Engine {
 public:
  explicit Engine(cudaStream_t s) : s_(s), flag_(sizeof(int) * 4, s) {}
  cudaStream_t stream() const { return s_; }
  Stats& stats() { return st_; }

  // precision of the large contractions (0 = FP64, 1 = 3xTF32, 2 = BF16x3, 3 = BF16x6,
  // 4 = Ozaki slices); FP64 and the Ozaki slices are float64-grade, the others float-grade
  int prec = 0;
  bool fp64_grade() const { return prec == 0 || prec == 4; }
  bool allow_tc = true;

  void gemm(const GemmDesc& d, const double* A, const double* B, double* C);
  // C = A Omega with the Gaussian sketch Omega generated while the tensor-core operand is
  // packed (never stored).  Only for contractions that take the split-precision path;
  // returns false, having done nothing, otherwise.
  bool gemm_gauss_b(const GemmDesc& d, const double* A, const GaussSrc& g, double* C);
  // row-major C (M x N) = alpha op(A) op(B) + beta C, op = transpose when flag set;
  // lda etc. are the row lengths of the stored matrices.
  void mm(int64_t M, int64_t N, int64_t K, const double* A, int64_t lda, bool ta,
          const double* B, int64_t ldb, bool tb, double* C, int64_t ldc, double alpha = 1.0,
          double beta = 0.0);

  OrthResult orth(const double* Y, int64_t m, int64_t n);
  SvdResult svd(const double* A, int64_t m, int64_t n);

  // Randomized SVD of an implicit rows x cols operator: apply(X, w, Y) computes
  // Y = M X for X (cols x w), rapply(X, w, Z) computes Z = M^T X for X (rows x w).
  using Op = std::function<void(const double*, int64_t, double*)>;
  SvdResult rsvd(const Op& apply, const Op& rapply, int64_t rows, int64_t cols, int64_t ell,
                 int q, const double* omega);
  // Subspace iteration on a PSD rho (n x n, row-major): returns leading Ritz values in
  // S and vectors in U (n x k).
  SvdResult rsvd_psd(const double* rho, int64_t n, int64_t ell, int q, const double* omega);

  // Orthonormal basis of an implicit panel Q = L X whose rows are never formed: only the
  // metric G = L^T L is available, as metric(V, w, U) computing U = G V for V (nin x w).
  // CholeskyQR2 (shifted CholeskyQR3 for split precision) on the small Grams X^T G X.
  // Returns V (the new basis is Q = L V), U = G V and R with L X = Q R; ok = false when a
  // Cholesky factorisation breaks down (rank deficiency).
  struct MetricOrth {
    DMat V, U, R;
    int k = 0;
    bool ok = false;
  };
  MetricOrth orth_metric(const double* X, int64_t nin, int64_t w, const Op& metric);

  // Forward-mode (tangent) rules, in tangent.cu.  grp[i] is the multiplet id of singular
  // value i: pairs inside one multiplet get no mutual rotation.
  struct SvdTan {
    DMat U, V;              // tangents of the leading kt columns of U (m x kt) and V (n x kt)
    std::vector<double> s;  // tangents of the leading kt singular values
  };
  SvdTan svd_tan(const double* Ad, int64_t m, int64_t n, const SvdResult& e, int kt,
                 const std::vector<int>& grp);
  struct OrthT {
    OrthResult o;
    DMat Qd, Rd;
  };
  // FP64 orth (CholeskyQR2, rank-revealing SVD fallback) with the tangents of Q and R
  OrthT orth_t(const double* Y, const double* Yd, int64_t m, int64_t n, double tau);
  struct RsvdT {
    SvdResult e;
    SvdTan t;
  };
  // rsvd / rsvd_psd with tangents; apply_d and rapply_d apply dM and dM^T
  RsvdT rsvd_t(const Op& apply, const Op& rapply, const Op& apply_d, const Op& rapply_d,
               int64_t rows, int64_t cols, int64_t ell, int q, const double* omega, double tau);
  RsvdT rsvd_psd_t(const double* rho, const double* rho_d, int64_t n, int64_t ell, int q,
                   const double* omega, double tau);
  DevBuf polar_tan(const SvdResult& e, const double* Gd, int m);
  DevBuf upload(const std::vector<double>& v);

  std::vector<double> to_host(const double* p, int64_t n);
  int read_flag(int idx = 0);
  int* flag(int idx = 0) { return flag_.as<int>() + idx; }
  double* scratch_double() { return reinterpret_cast<double*>(flag_.as<int>() + 2); }

 private:
  OrthResult cholqr2(const double* Y, int64_t m, int64_t n, double shift, bool& ok);
  cudaStream_t s_;
  Stats st_;
  DevBuf flag_;
};

int keep_count(const std::vector<double>& v, double rel, int64_t cap);
// multiplet id of each value of a descending sequence (gap <= tau times the larger value)
std::vector<int> multiplet_groups(const std::vector<double>& v, double tau);
// tangent.cu: y += a x;  x *= v^p with dx <- dx v^p + p x v^(p-1) dv;  dT/dtheta of Ising T
void axpy(double* y, const double* x, int64_t n, double a, cudaStream_t s);
void scale_axis_tan(double* x, double* dx, const double* v, const double* dv, int64_t outer,
                    int64_t n, int64_t inner, int power, cudaStream_t s);
void ising_tensor_tan(double beta, double h, int d, int dir, double* dT, cudaStream_t s);

}  // namespace tatrg
