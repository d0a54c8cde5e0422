#include "engine.cuh"

#include <cmath>

namespace tatrg {

int keep_count(const std::vector<double>& v, double rel, int64_t cap) {
  if (v.empty() || !(v[0] > 0.0)) return 0;
  int64_t n = 0;
  for (double x : v) n += (x > rel * v[0]) ? 1 : 0;
  if (cap > 0) n = std::min(n, cap);
  return int(n);
}

// Tensor cores for the large contractions of the split forms; the FP64 CUDA-core kernel
// for everything small (where 128-row tiles would be mostly padding).
static bool use_tc(const Engine& e, const GemmDesc& d) {
  const double M = double(d.m.total()), N = double(d.n.total()), K = double(d.k.total());
  return e.prec != 0 && e.allow_tc && tc_available() && M * N * K >= 2.0e7 && M >= 32 &&
         N >= 16 && K >= 16;
}

void Engine::gemm(const GemmDesc& d, const double* A, const double* B, double* C) {
  if (use_tc(*this, d) && prec == 4) gemm_oz(d, A, B, C, s_, &st_);
  else if (use_tc(*this, d)) gemm_tc(d, A, B, C, prec, s_, &st_);
  else gemm_f64(d, A, B, C, s_, &st_);
}

bool Engine::gemm_gauss_b(const GemmDesc& d, const double* A, const GaussSrc& g, double* C) {
  if (!use_tc(*this, d) || prec == 4) return false;  // the Ozaki slices read a stored sketch
  gemm_tc(d, A, nullptr, C, prec, s_, &st_, &g);
  return true;
}

void Engine::mm(int64_t M, int64_t N, int64_t K, const double* A, int64_t lda, bool ta,
                const double* B, int64_t ldb, bool tb, double* C, int64_t ldc, double alpha,
                double beta) {
  GemmDesc g;
  g.m = modes({{M, ta ? 1 : lda, ldc}});
  g.n = modes({{N, tb ? ldb : 1, 1}});
  g.k = modes({{K, ta ? lda : 1, tb ? 1 : ldb}});
  g.alpha = alpha;
  g.beta = beta;
  gemm(g, A, B, C);
}

std::vector<double> Engine::to_host(const double* p, int64_t n) {
  std::vector<double> h(size_t(std::max<int64_t>(n, 0)));
  if (n > 0) TATRG_CUDA(cudaMemcpyAsync(h.data(), p, n * sizeof(double), cudaMemcpyDeviceToHost, s_));
  TATRG_CUDA(cudaStreamSynchronize(s_));
  return h;
}

int Engine::read_flag(int idx) {
  int v = 0;
  TATRG_CUDA(cudaMemcpyAsync(&v, flag_.as<int>() + idx, sizeof(int), cudaMemcpyDeviceToHost, s_));
  TATRG_CUDA(cudaStreamSynchronize(s_));
  return v;
}

// CholeskyQR2 (Yamamoto et al. 2015), optionally with a shifted first pass (shifted
// CholeskyQR3, Fukaya et al. 2020): Q = Y R^-1, R = R2 R1.  ok = false on breakdown.
OrthResult Engine::cholqr2(const double* Y, int64_t m, int64_t n, double shift, bool& ok) {
  OrthResult out;
  const int passes = shift > 0.0 ? 3 : 2;
  DevBuf G(n * n * sizeof(double), s_), Rk(n * n * sizeof(double), s_),
      Ri(n * n * sizeof(double), s_), Racc(n * n * sizeof(double), s_),
      Rtmp(n * n * sizeof(double), s_);
  DMat cur;
  const double* src = Y;
  for (int pass = 0; pass < passes; ++pass) {
    mm(n, n, m, src, n, true, src, n, false, G.d(), n);
    cholesky(G.d(), int(n), Rk.d(), flag(0), pass == 0 ? shift : 0.0, s_);
    st_.launches++;
    if (read_flag(0) != 0) { ok = false; return out; }
    tri_inverse(Rk.d(), int(n), Ri.d(), s_);
    st_.launches++;
    DMat nxt;
    nxt.buf = dalloc(m * n, s_);
    nxt.rows = m;
    nxt.cols = n;
    mm(m, n, n, src, n, false, Ri.d(), n, false, nxt.p(), n);
    if (pass == 0) {
      TATRG_CUDA(cudaMemcpyAsync(Racc.d(), Rk.d(), n * n * sizeof(double), cudaMemcpyDeviceToDevice, s_));
    } else {
      mm(n, n, n, Rk.d(), n, false, Racc.d(), n, false, Rtmp.d(), n);
      std::swap(Racc, Rtmp);
    }
    cur = std::move(nxt);
    src = cur.p();
  }
  ok = true;
  out.Q = std::move(cur);
  out.R.buf = std::move(Racc);
  out.R.rows = n;
  out.R.cols = n;
  out.k = int(n);
  return out;
}

OrthResult Engine::orth(const double* Y, int64_t m, int64_t n) {
  TATRG_CHECK(n >= 1, TATRG_EINVAL, "orth: empty matrix");
  bool ok = false;
  OrthResult r;
  if (m >= n && n <= cholesky_max_n()) {
    // FP64 Grams: plain CholeskyQR2.  Split-precision Grams carry ~1e-7 relative error, so
    // their first pass is shifted (shifted CholeskyQR3).
    r = cholqr2(Y, m, n, fp64_grade() ? 0.0 : 1e-6, ok);
    if (ok) return r;
  }
  // Rank-revealing fallback: one-sided Jacobi SVD of Y itself (no squared condition
  // number), Y = U S V^T; keep the directions above the rounding floor: Q = U_k,
  // R = S_k V_k^T.
  SvdResult e = svd(Y, m, n);
  const double cut = fp64_grade() ? 1e-14 : 1e-7;
  int k = keep_count(e.s, cut, std::min(m, n));
  TATRG_CHECK(k >= 1, TATRG_ENUMERIC, "orth: zero matrix");
  OrthResult out;
  out.Q.buf = dalloc(m * k, s_);
  out.Q.rows = m;
  out.Q.cols = k;
  copy_modes(out.Q.p(), e.U.p(), modes({{m, e.U.cols, k}, {k, 1, 1}}), 1.0, s_);
  out.R.buf = dalloc(int64_t(k) * n, s_);
  out.R.rows = k;
  out.R.cols = n;
  copy_modes(out.R.p(), e.V.p(), modes({{k, 1, n}, {n, e.V.cols, 1}}), 1.0, s_);  // V_k^T
  scale_axis(out.R.p(), e.S.d(), 1, k, n, 1, s_);
  out.k = k;
  return out;
}

Engine::MetricOrth Engine::orth_metric(const double* X, int64_t nin, int64_t w, const Op& metric) {
  MetricOrth out;
  if (w > cholesky_max_n()) return out;  // ok = false: the caller takes the explicit path
  const int passes = fp64_grade() ? 2 : 3;
  const double shift = fp64_grade() ? 0.0 : 1e-6;
  DevBuf G(w * w * sizeof(double), s_), Rk(w * w * sizeof(double), s_), Ri(w * w * sizeof(double), s_),
      Racc(w * w * sizeof(double), s_), Rtmp(w * w * sizeof(double), s_);
  DMat cur;
  cur.buf = dalloc(nin * w, s_);
  cur.rows = nin;
  cur.cols = w;
  TATRG_CUDA(cudaMemcpyAsync(cur.p(), X, nin * w * sizeof(double), cudaMemcpyDeviceToDevice, s_));
  DMat U;
  U.buf = dalloc(nin * w, s_);
  U.rows = nin;
  U.cols = w;
  for (int pass = 0; pass < passes; ++pass) {
    metric(cur.p(), w, U.p());
    mm(w, w, nin, cur.p(), w, true, U.p(), w, false, G.d(), w);
    cholesky(G.d(), int(w), Rk.d(), flag(0), pass == 0 ? shift : 0.0, s_);
    st_.launches++;
    if (read_flag(0) != 0) return out;  // ok = false
    tri_inverse(Rk.d(), int(w), Ri.d(), s_);
    st_.launches++;
    DMat nxt;
    nxt.buf = dalloc(nin * w, s_);
    nxt.rows = nin;
    nxt.cols = w;
    mm(nin, w, w, cur.p(), w, false, Ri.d(), w, false, nxt.p(), w);
    if (pass == 0) {
      TATRG_CUDA(cudaMemcpyAsync(Racc.d(), Rk.d(), w * w * sizeof(double), cudaMemcpyDeviceToDevice, s_));
    } else {
      mm(w, w, w, Rk.d(), w, false, Racc.d(), w, false, Rtmp.d(), w);
      std::swap(Racc, Rtmp);
    }
    cur = std::move(nxt);
  }
  metric(cur.p(), w, U.p());  // U = G V for the final basis
  out.V = std::move(cur);
  out.U = std::move(U);
  out.R.buf = std::move(Racc);
  out.R.rows = w;
  out.R.cols = w;
  out.k = int(w);
  out.ok = true;
  return out;
}

SvdResult Engine::svd(const double* A, int64_t m, int64_t n) {
  SvdResult r;
  const int64_t k = std::min(m, n);
  r.S = DevBuf(k * sizeof(double), s_);
  if (m >= n) {
    r.U.buf = dalloc(m * n, s_);
    r.U.rows = m;
    r.U.cols = n;
    r.V.buf = dalloc(n * n, s_);
    r.V.rows = n;
    r.V.cols = n;
    if (qrcp_svd_fits(m, int(n))) jacobi_svd_qrcp(A, m, int(n), r.U.p(), r.S.d(), r.V.p(), flag(1), s_, &st_);
    else jacobi_svd(A, m, int(n), r.U.p(), r.S.d(), r.V.p(), flag(1), s_, &st_);
  } else {
    DevBuf At(m * n * sizeof(double), s_);
    transpose(A, m, n, At.d(), s_);
    r.V.buf = dalloc(n * m, s_);
    r.V.rows = n;
    r.V.cols = m;
    r.U.buf = dalloc(m * m, s_);
    r.U.rows = m;
    r.U.cols = m;
    if (qrcp_svd_fits(n, int(m))) jacobi_svd_qrcp(At.d(), n, int(m), r.V.p(), r.S.d(), r.U.p(), flag(1), s_, &st_);
    else jacobi_svd(At.d(), n, int(m), r.V.p(), r.S.d(), r.U.p(), flag(1), s_, &st_);
  }
  r.r = int(k);
  r.s = to_host(r.S.d(), k);
  const int jst = read_flag(1);
  TATRG_CHECK(jst != 2, TATRG_ETIMEOUT, "Jacobi SVD: a grid barrier timed out");
  TATRG_CHECK(jst == 0, TATRG_ENUMERIC, "Jacobi SVD did not converge");
  for (double x : r.s) TATRG_CHECK(std::isfinite(x), TATRG_ENUMERIC, "non-finite singular value");
  return r;
}

SvdResult Engine::rsvd(const Op& apply, const Op& rapply, int64_t rows, int64_t cols,
                       int64_t ell, int q, const double* omega) {
  DMat Y;
  Y.buf = dalloc(rows * ell, s_);
  apply(omega, ell, Y.p());
  OrthResult Q = orth(Y.p(), rows, ell);
  for (int it = 0; it < q; ++it) {
    DMat Z;
    Z.buf = dalloc(cols * Q.k, s_);
    rapply(Q.Q.p(), Q.k, Z.p());
    OrthResult Qt = orth(Z.p(), cols, Q.k);
    DMat Y2;
    Y2.buf = dalloc(rows * Qt.k, s_);
    apply(Qt.Q.p(), Qt.k, Y2.p());
    Q = orth(Y2.p(), rows, Qt.k);
  }
  DMat Bt;
  Bt.buf = dalloc(cols * Q.k, s_);
  rapply(Q.Q.p(), Q.k, Bt.p());          // (Q^T M)^T
  OrthResult P = orth(Bt.p(), cols, Q.k); // Bt = P R, R: kp x kq
  const int64_t kq = Q.k, kp = P.k;
  DevBuf Rt(kq * kp * sizeof(double), s_);
  transpose(P.R.p(), kp, kq, Rt.d(), s_);  // R^T: kq x kp
  SvdResult c = svd(Rt.d(), kq, kp);       // R^T = W S Z^T
  const int64_t r = c.r;
  SvdResult out;
  out.r = int(r);
  out.s = c.s;
  out.S = std::move(c.S);
  out.U.buf = dalloc(rows * r, s_);
  out.U.rows = rows;
  out.U.cols = r;
  mm(rows, r, kq, Q.Q.p(), kq, false, c.U.p(), c.U.cols, false, out.U.p(), r);
  out.V.buf = dalloc(cols * r, s_);
  out.V.rows = cols;
  out.V.cols = r;
  mm(cols, r, kp, P.Q.p(), kp, false, c.V.p(), c.V.cols, false, out.V.p(), r);
  return out;
}

SvdResult Engine::rsvd_psd(const double* rho, int64_t n, int64_t ell, int q, const double* omega) {
  auto app = [&](const double* X, int64_t w, double* Yo) {
    mm(n, w, n, rho, n, false, X, w, false, Yo, w);
  };
  DMat Y;
  Y.buf = dalloc(n * ell, s_);
  app(omega, ell, Y.p());
  OrthResult Q = orth(Y.p(), n, ell);
  for (int it = 0; it < q; ++it) {
    DMat Z;
    Z.buf = dalloc(n * Q.k, s_);
    app(Q.Q.p(), Q.k, Z.p());
    OrthResult Qt = orth(Z.p(), n, Q.k);
    DMat Y2;
    Y2.buf = dalloc(n * Qt.k, s_);
    app(Qt.Q.p(), Qt.k, Y2.p());
    Q = orth(Y2.p(), n, Qt.k);
  }
  const int64_t k = Q.k;
  DMat RQ;
  RQ.buf = dalloc(n * k, s_);
  app(Q.Q.p(), k, RQ.p());
  DevBuf Bm(k * k * sizeof(double), s_);
  mm(k, k, n, Q.Q.p(), k, true, RQ.p(), k, false, Bm.d(), k);  // Q^T rho Q
  SvdResult e = svd(Bm.d(), k, k);
  SvdResult out;
  out.r = e.r;
  out.s = e.s;
  out.S = std::move(e.S);
  out.U.buf = dalloc(n * e.r, s_);
  out.U.rows = n;
  out.U.cols = e.r;
  mm(n, e.r, k, Q.Q.p(), k, false, e.V.p(), e.V.cols, false, out.U.p(), e.r);
  return out;
}

}  // namespace tatrg
