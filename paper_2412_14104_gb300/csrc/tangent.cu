// Forward-mode (tangent) rules of the factorisations in the RG step.  With two scalar
// inputs (beta, h) the derivative of ln Z / V is one tangent pass per input, run beside
// the primal step: every contraction C = A B carries dC = dA B + A dB, and the rules below
// carry the tangents through the QR, the SVD, the randomized SVDs and the gauge rules.
//
//   SVD  A = U S V^T (m >= n), J = U^T dA V:
//     dS_j = J_jj,
//     dU_j = sum_{i != j} U_i (J_ij s_j + J_ji s_i) / (s_j^2 - s_i^2) + (1 - U U^T) dA V_j / s_j,
//     dV_j = sum_{i != j} V_i (J_ij s_i + J_ji s_j) / (s_j^2 - s_i^2).
//     Pairs inside one degenerate multiplet get no mutual rotation: the basis of a
//     multiplet is fixed afterwards by a gauge rule whose result depends only on the
//     multiplet's subspace, so that component does not reach the output.
//   QR  Y = Q R (R upper, positive diagonal), C = Q^T dY R^-1, X = upper part of C with
//     the strict upper part doubled:  dR = X R,  dQ = dY R^-1 - Q X.
//   Polar factor O = U_g V_g^T of G = U_g S_g V_g^T:  L = U_g^T dG V_g,
//     dO = U_g W V_g^T with W_ij = (L_ij - L_ji) / (s_i + s_j).
#include "engine.cuh"

#include <cmath>

namespace tatrg {

namespace {
__global__ void svd_tan_coef_kernel(const double* J, const double* s, const int* grp, int n,
                                    int k, double* Xu, double* Xv, double* sdot) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * k; e += gridDim.x * blockDim.x) {
    const int i = e / k, j = e - (e / k) * k;
    const double jij = J[int64_t(i) * n + j], jji = J[int64_t(j) * n + i];
    const double si = s[i], sj = s[j];
    double u = -jij / sj, v = 0.0;
    if (i != j && grp[i] != grp[j]) {
      const double den = (sj - si) * (sj + si);
      u += (jij * sj + jji * si) / den;
      v = (jij * si + jji * sj) / den;
    }
    if (i == j) {
      u = -jij / sj;
      sdot[j] = jij;
    }
    Xu[e] = u;
    Xv[e] = v;
  }
}

// X = upper part of C with the strict upper part C_ij + C_ji
__global__ void qr_tan_kernel(const double* C, int n, double* X) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) {
    const int i = e / n, j = e - (e / n) * n;
    X[e] = i > j ? 0.0 : (i == j ? C[e] : C[e] + C[int64_t(j) * n + i]);
  }
}

__global__ void polar_tan_kernel(const double* L, const double* s, int m, double* W) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * m; e += gridDim.x * blockDim.x) {
    const int i = e / m, j = e - (e / m) * m;
    W[e] = (L[e] - L[int64_t(j) * m + i]) / (s[i] + s[j]);
  }
}

__global__ void axpy_kernel(double* y, const double* x, int64_t n, double a) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n;
       e += int64_t(gridDim.x) * blockDim.x)
    y[e] = fma(a, x[e], y[e]);
}

// x[o, a, i] *= v_a^p and its tangent dx <- dx v^p + p x v^(p-1) dv (p = 1 or 2), in place
__global__ void scale_axis_tan_kernel(double* x, double* dx, const double* v, const double* dv,
                                      int64_t outer, int64_t n, int64_t inner, int p) {
  const int64_t total = outer * n * inner;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t a = (e / inner) % n;
    const double va = v[a], xa = x[e];
    const double vp = p == 2 ? va * va : va;
    const double dvp = p == 2 ? 2.0 * va * dv[a] : dv[a];
    dx[e] = dx[e] * vp + xa * dvp;
    x[e] = xa * vp;
  }
}

// d/dtheta of the Ising tensor (theta = beta for dir 0, h for dir 1), same layout as T
__global__ void ising_tensor_tan_kernel(double beta, double h, int d, int dir, double* dT) {
  const int n = 1 << (2 * d);
  const double c = sqrt(2.0 * cosh(beta)), sn = sqrt(2.0 * sinh(beta));
  // W = U diag(c, sn) U^T, U = [[1, 1], [1, -1]] / sqrt(2); dW/dbeta from dc, dsn
  const double dc = sinh(beta) / c, dsn = cosh(beta) / sn;
  double w[2][2], dw[2][2];
  w[0][0] = w[1][1] = 0.5 * (c + sn);
  w[0][1] = w[1][0] = 0.5 * (c - sn);
  dw[0][0] = dw[1][1] = 0.5 * (dc + dsn);
  dw[0][1] = dw[1][0] = 0.5 * (dc - dsn);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int si = 0; si < 2; ++si) {
      const double sg = si == 0 ? 1.0 : -1.0;
      const double eh = exp(sg * h);
      double prod = 1.0, dprod = 0.0;  // product over legs and its beta derivative
      for (int leg = 0; leg < 2 * d; ++leg) {
        const int x = (e >> (2 * d - 1 - leg)) & 1;
        dprod = dprod * w[si][x] + prod * dw[si][x];
        prod *= w[si][x];
      }
      acc += dir == 0 ? eh * dprod : sg * eh * prod;
    }
    dT[e] = acc;
  }
}

int blocks_for(int64_t n) { return int(std::max<int64_t>(1, std::min<int64_t>(cdiv(n, 256), int64_t(sm_count()) * 16))); }
}  // namespace

std::vector<int> multiplet_groups(const std::vector<double>& v, double tau) {
  std::vector<int> g(v.size(), 0);
  for (size_t i = 1; i < v.size(); ++i)
    g[i] = (v[i - 1] - v[i] > tau * v[i - 1]) ? g[i - 1] + 1 : g[i - 1];
  return g;
}

void axpy(double* y, const double* x, int64_t n, double a, cudaStream_t s) {
  if (n <= 0) return;
  check_extent(y, n - 1, sizeof(double), "axpy y");
  check_extent(x, n - 1, sizeof(double), "axpy x");
  axpy_kernel<<<blocks_for(n), 256, 0, s>>>(y, x, n, a);
  TATRG_CUDA(cudaGetLastError());
}

void scale_axis_tan(double* x, double* dx, const double* v, const double* dv, int64_t outer,
                    int64_t n, int64_t inner, int power, cudaStream_t s) {
  TATRG_CHECK(power == 1 || power == 2, TATRG_EINVAL, "scale_axis_tan: power must be 1 or 2");
  const int64_t total = outer * n * inner;
  if (total == 0) return;
  check_extent(x, total - 1, sizeof(double), "scale_axis_tan x");
  check_extent(dx, total - 1, sizeof(double), "scale_axis_tan dx");
  scale_axis_tan_kernel<<<blocks_for(total), 256, 0, s>>>(x, dx, v, dv, outer, n, inner, power);
  TATRG_CUDA(cudaGetLastError());
}

void ising_tensor_tan(double beta, double h, int d, int dir, double* dT, cudaStream_t s) {
  ising_tensor_tan_kernel<<<blocks_for(int64_t(1) << (2 * d)), 256, 0, s>>>(beta, h, d, dir, dT);
  TATRG_CUDA(cudaGetLastError());
}

DevBuf Engine::upload(const std::vector<double>& v) {
  DevBuf b(std::max<size_t>(v.size(), 1) * sizeof(double), s_);
  if (!v.empty())
    TATRG_CUDA(cudaMemcpyAsync(b.d(), v.data(), v.size() * sizeof(double), cudaMemcpyHostToDevice, s_));
  return b;
}

// Tangent of the leading kt singular triplets of A (m x n) given its SVD e from svd().
Engine::SvdTan Engine::svd_tan(const double* Ad, int64_t m, int64_t n, const SvdResult& e,
                               int kt, const std::vector<int>& grp) {
  SvdTan t;
  // Work on the tall orientation: A' = A (m >= n) or A^T (m < n), A' = U' S V'^T.
  const bool tall = m >= n;
  const int64_t M = tall ? m : n, N = tall ? n : m;
  const DMat& Up = tall ? e.U : e.V;  // M x N
  const DMat& Vp = tall ? e.V : e.U;  // N x N
  TATRG_CHECK(kt >= 0 && kt <= N && int64_t(grp.size()) >= N, TATRG_EINVAL, "svd_tan: bad sizes");
  t.U.rows = m;
  t.V.rows = n;
  t.U.cols = t.V.cols = kt;
  t.U.buf = dalloc(m * kt, s_);
  t.V.buf = dalloc(n * kt, s_);
  t.s.assign(kt, 0.0);
  if (kt == 0) return t;
  // T1 = A'_dot V' (M x N), J = U'^T T1 (N x N)
  DevBuf T1(M * N * sizeof(double), s_), J(N * N * sizeof(double), s_);
  if (tall) mm(M, N, N, Ad, n, false, Vp.p(), Vp.cols, false, T1.d(), N);
  else mm(M, N, N, Ad, n, true, Vp.p(), Vp.cols, false, T1.d(), N);
  mm(N, N, M, Up.p(), Up.cols, true, T1.d(), N, false, J.d(), N);
  std::vector<int> g(grp.begin(), grp.begin() + N);
  DevBuf gd(N * sizeof(int), s_), Xu(N * kt * sizeof(double), s_), Xv(N * kt * sizeof(double), s_),
      sd(kt * sizeof(double), s_);
  TATRG_CUDA(cudaMemcpyAsync(gd.d(), g.data(), N * sizeof(int), cudaMemcpyHostToDevice, s_));
  svd_tan_coef_kernel<<<blocks_for(N * kt), 256, 0, s_>>>(J.d(), e.S.d(), gd.as<int>(), int(N), kt,
                                                          Xu.d(), Xv.d(), sd.d());
  TATRG_CUDA(cudaGetLastError());
  st_.launches++;
  // dU' = U' Xu + T1[:, :kt] / s,  dV' = V' Xv
  DMat& dUp = tall ? t.U : t.V;
  DMat& dVp = tall ? t.V : t.U;
  copy_modes(dUp.p(), T1.d(), modes({{M, N, kt}, {kt, 1, 1}}), 1.0, s_);
  std::vector<double> inv(kt);
  for (int j = 0; j < kt; ++j) inv[j] = 1.0 / e.s[j];
  DevBuf invd = upload(inv);
  scale_axis(dUp.p(), invd.d(), M, kt, 1, 1, s_);
  mm(M, kt, N, Up.p(), Up.cols, false, Xu.d(), kt, false, dUp.p(), kt, 1.0, 1.0);
  mm(N, kt, N, Vp.p(), Vp.cols, false, Xv.d(), kt, false, dVp.p(), kt);
  t.s = to_host(sd.d(), kt);
  return t;
}

Engine::OrthT Engine::orth_t(const double* Y, const double* Yd, int64_t m, int64_t n, double tau) {
  OrthT out;
  bool ok = false;
  if (m >= n) out.o = cholqr2(Y, m, n, 0.0, ok);
  if (ok) {
    DevBuf Ri(n * n * sizeof(double), s_), C(n * n * sizeof(double), s_), X(n * n * sizeof(double), s_);
    tri_inverse(out.o.R.p(), int(n), Ri.d(), s_);
    st_.launches++;
    out.Qd.buf = dalloc(m * n, s_);
    out.Qd.rows = m;
    out.Qd.cols = n;
    mm(m, n, n, Yd, n, false, Ri.d(), n, false, out.Qd.p(), n);          // dY R^-1
    mm(n, n, m, out.o.Q.p(), n, true, out.Qd.p(), n, false, C.d(), n);  // C
    qr_tan_kernel<<<blocks_for(n * n), 256, 0, s_>>>(C.d(), int(n), X.d());
    TATRG_CUDA(cudaGetLastError());
    st_.launches++;
    mm(m, n, n, out.o.Q.p(), n, false, X.d(), n, false, out.Qd.p(), n, -1.0, 1.0);
    out.Rd.buf = dalloc(n * n, s_);
    out.Rd.rows = out.Rd.cols = n;
    mm(n, n, n, X.d(), n, false, out.o.R.p(), n, false, out.Rd.p(), n);
    return out;
  }
  // rank-revealing fallback, as in orth(): Q = U_k, R = S_k V_k^T
  SvdResult e = svd(Y, m, n);
  const int k = keep_count(e.s, 1e-14, std::min(m, n));
  TATRG_CHECK(k >= 1, TATRG_ENUMERIC, "orth: zero matrix");
  SvdTan t = svd_tan(Yd, m, n, e, k, multiplet_groups(e.s, tau));
  OrthResult& o = out.o;
  o.Q.buf = dalloc(m * k, s_);
  o.Q.rows = m;
  o.Q.cols = k;
  copy_modes(o.Q.p(), e.U.p(), modes({{m, e.U.cols, k}, {k, 1, 1}}), 1.0, s_);
  o.R.buf = dalloc(int64_t(k) * n, s_);
  o.R.rows = k;
  o.R.cols = n;
  copy_modes(o.R.p(), e.V.p(), modes({{k, 1, n}, {n, e.V.cols, 1}}), 1.0, s_);
  scale_axis(o.R.p(), e.S.d(), 1, k, n, 1, s_);
  o.k = k;
  out.Qd = std::move(t.U);
  // dR = diag(ds) V_k^T + S_k dV_k^T
  out.Rd.buf = dalloc(int64_t(k) * n, s_);
  out.Rd.rows = k;
  out.Rd.cols = n;
  copy_modes(out.Rd.p(), t.V.p(), modes({{k, 1, n}, {n, k, 1}}), 1.0, s_);
  scale_axis(out.Rd.p(), e.S.d(), 1, k, n, 1, s_);
  DevBuf tmp(int64_t(k) * n * sizeof(double), s_), dsd = upload(t.s);
  copy_modes(tmp.d(), e.V.p(), modes({{k, 1, n}, {n, e.V.cols, 1}}), 1.0, s_);
  scale_axis(tmp.d(), dsd.d(), 1, k, n, 1, s_);
  axpy(out.Rd.p(), tmp.d(), int64_t(k) * n, 1.0, s_);
  return out;
}

Engine::RsvdT Engine::rsvd_t(const Op& apply, const Op& rapply, const Op& apply_d,
                             const Op& rapply_d, int64_t rows, int64_t cols, int64_t ell, int q,
                             const double* omega, double tau) {
  // Y = M Omega, dY = dM Omega
  DMat Y, Yd;
  Y.buf = dalloc(rows * ell, s_);
  Yd.buf = dalloc(rows * ell, s_);
  apply(omega, ell, Y.p());
  apply_d(omega, ell, Yd.p());
  OrthT Q = orth_t(Y.p(), Yd.p(), rows, ell, tau);
  // Z = M^T Q, dZ = dM^T Q + M^T dQ (and the same shape for M Q)
  auto both = [&](const Op& f, const Op& fd, const OrthT& B, int64_t len, DMat& Z, DMat& Zd) {
    const int64_t k = B.o.k;
    Z.buf = dalloc(len * k, s_);
    Zd.buf = dalloc(len * k, s_);
    DevBuf tmp(len * k * sizeof(double), s_);
    f(B.o.Q.p(), k, Z.p());
    fd(B.o.Q.p(), k, Zd.p());
    f(B.Qd.p(), k, tmp.d());
    axpy(Zd.p(), tmp.d(), len * k, 1.0, s_);
  };
  for (int it = 0; it < q; ++it) {
    DMat Z, Zd;
    both(rapply, rapply_d, Q, cols, Z, Zd);
    OrthT Qt = orth_t(Z.p(), Zd.p(), cols, Q.o.k, tau);
    DMat Y2, Y2d;
    both(apply, apply_d, Qt, rows, Y2, Y2d);
    Q = orth_t(Y2.p(), Y2d.p(), rows, Qt.o.k, tau);
  }
  DMat Bt, Btd;
  both(rapply, rapply_d, Q, cols, Bt, Btd);  // (Q^T M)^T
  const int64_t kq = Q.o.k;
  OrthT P = orth_t(Bt.p(), Btd.p(), cols, kq, tau);  // Bt = P R
  const int64_t kp = P.o.k;
  DevBuf Rt(kq * kp * sizeof(double), s_), Rtd(kq * kp * sizeof(double), s_);
  transpose(P.o.R.p(), kp, kq, Rt.d(), s_);
  transpose(P.Rd.p(), kp, kq, Rtd.d(), s_);
  SvdResult c = svd(Rt.d(), kq, kp);  // R^T = W S Z^T
  const int kt = keep_count(c.s, 1e-14, c.r);
  SvdTan ct = svd_tan(Rtd.d(), kq, kp, c, kt, multiplet_groups(c.s, tau));
  RsvdT out;
  const int64_t r = c.r;
  out.e.r = int(r);
  out.e.s = c.s;
  out.e.S = std::move(c.S);
  out.e.U.buf = dalloc(rows * r, s_);
  out.e.U.rows = rows;
  out.e.U.cols = r;
  mm(rows, r, kq, Q.o.Q.p(), kq, false, c.U.p(), c.U.cols, false, out.e.U.p(), r);
  out.e.V.buf = dalloc(cols * r, s_);
  out.e.V.rows = cols;
  out.e.V.cols = r;
  mm(cols, r, kp, P.o.Q.p(), kp, false, c.V.p(), c.V.cols, false, out.e.V.p(), r);
  // dU = dQ W + Q dW, dV = dP Z + P dZ  (first kt columns)
  out.t.s = ct.s;
  out.t.U.buf = dalloc(rows * kt, s_);
  out.t.U.rows = rows;
  out.t.U.cols = kt;
  out.t.V.buf = dalloc(cols * kt, s_);
  out.t.V.rows = cols;
  out.t.V.cols = kt;
  if (kt > 0) {
    mm(rows, kt, kq, Q.Qd.p(), kq, false, c.U.p(), c.U.cols, false, out.t.U.p(), kt);
    mm(rows, kt, kq, Q.o.Q.p(), kq, false, ct.U.p(), kt, false, out.t.U.p(), kt, 1.0, 1.0);
    mm(cols, kt, kp, P.Qd.p(), kp, false, c.V.p(), c.V.cols, false, out.t.V.p(), kt);
    mm(cols, kt, kp, P.o.Q.p(), kp, false, ct.V.p(), kt, false, out.t.V.p(), kt, 1.0, 1.0);
  }
  return out;
}

Engine::RsvdT Engine::rsvd_psd_t(const double* rho, const double* rho_d, int64_t n, int64_t ell,
                                 int q, const double* omega, double tau) {
  auto app = [&](const double* R, const double* X, int64_t w, double* Yo, double beta) {
    mm(n, w, n, R, n, false, X, w, false, Yo, w, 1.0, beta);
  };
  // Z = rho X, dZ = drho X + rho dX
  auto both = [&](const double* X, const double* Xd, int64_t w, DMat& Z, DMat& Zd) {
    Z.buf = dalloc(n * w, s_);
    Zd.buf = dalloc(n * w, s_);
    app(rho, X, w, Z.p(), 0.0);
    app(rho_d, X, w, Zd.p(), 0.0);
    if (Xd) app(rho, Xd, w, Zd.p(), 1.0);
  };
  DMat Y, Yd;
  both(omega, nullptr, ell, Y, Yd);
  OrthT Q = orth_t(Y.p(), Yd.p(), n, ell, tau);
  for (int it = 0; it < q; ++it) {
    DMat Z, Zd;
    both(Q.o.Q.p(), Q.Qd.p(), Q.o.k, Z, Zd);
    OrthT Qt = orth_t(Z.p(), Zd.p(), n, Q.o.k, tau);
    DMat Y2, Y2d;
    both(Qt.o.Q.p(), Qt.Qd.p(), Qt.o.k, Y2, Y2d);
    Q = orth_t(Y2.p(), Y2d.p(), n, Qt.o.k, tau);
  }
  const int64_t k = Q.o.k;
  DMat RQ, RQd;
  both(Q.o.Q.p(), Q.Qd.p(), k, RQ, RQd);
  // Bm = Q^T rho Q, dBm = dQ^T RQ + Q^T dRQ
  DevBuf Bm(k * k * sizeof(double), s_), Bmd(k * k * sizeof(double), s_);
  mm(k, k, n, Q.o.Q.p(), k, true, RQ.p(), k, false, Bm.d(), k);
  mm(k, k, n, Q.Qd.p(), k, true, RQ.p(), k, false, Bmd.d(), k);
  mm(k, k, n, Q.o.Q.p(), k, true, RQd.p(), k, false, Bmd.d(), k, 1.0, 1.0);
  SvdResult e = svd(Bm.d(), k, k);
  const int kt = keep_count(e.s, 1e-14, e.r);
  SvdTan et = svd_tan(Bmd.d(), k, k, e, kt, multiplet_groups(e.s, tau));
  RsvdT out;
  out.e.r = e.r;
  out.e.s = e.s;
  out.e.S = std::move(e.S);
  out.e.U.buf = dalloc(n * e.r, s_);
  out.e.U.rows = n;
  out.e.U.cols = e.r;
  mm(n, e.r, k, Q.o.Q.p(), k, false, e.V.p(), e.V.cols, false, out.e.U.p(), e.r);
  // dU = dQ V_e + Q dV_e
  out.t.s = et.s;
  out.t.U.buf = dalloc(n * kt, s_);
  out.t.U.rows = n;
  out.t.U.cols = kt;
  if (kt > 0) {
    mm(n, kt, k, Q.Qd.p(), k, false, e.V.p(), e.V.cols, false, out.t.U.p(), kt);
    mm(n, kt, k, Q.o.Q.p(), k, false, et.V.p(), kt, false, out.t.U.p(), kt, 1.0, 1.0);
  }
  return out;
}

// Tangent of the polar factor O of G (m x m) given G's SVD and dG; returns dO (m x m).
DevBuf Engine::polar_tan(const SvdResult& e, const double* Gd, int m) {
  DevBuf T(m * m * sizeof(double), s_), L(m * m * sizeof(double), s_), W(m * m * sizeof(double), s_),
      out(m * m * sizeof(double), s_);
  mm(m, m, m, Gd, m, false, e.V.p(), e.V.cols, false, T.d(), m);        // dG V
  mm(m, m, m, e.U.p(), e.U.cols, true, T.d(), m, false, L.d(), m);      // U^T dG V
  polar_tan_kernel<<<blocks_for(int64_t(m) * m), 256, 0, s_>>>(L.d(), e.S.d(), m, W.d());
  TATRG_CUDA(cudaGetLastError());
  st_.launches++;
  mm(m, m, m, e.U.p(), e.U.cols, false, W.d(), m, false, T.d(), m);     // U W
  mm(m, m, m, T.d(), m, false, e.V.p(), e.V.cols, true, out.d(), m);    // U W V^T
  return out;
}

}  // namespace tatrg
