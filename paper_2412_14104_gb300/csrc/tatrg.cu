// The Triad-ATRG RG step on the GPU (Sugimoto & Sasaki, arXiv:2412.14104, Sec. 2) and the
// C ABI of include/tatrg.h.  Every contraction below is one multi-mode GEMM whose modes
// are named after the paper's indices; stage order: bond swap (Eq. 1), triad isometries
// and tensors (Eqs. 2-4), squeezers (Eq. 5), contraction (Eqs. 6-7), re-split.
#include <cmath>
#include <cstring>
#include <atomic>
#include <mutex>
#include <thread>
#include <functional>
#include <exception>
#include <memory>
#include <string>

#include "engine.cuh"

using namespace tatrg;

namespace {

enum Stage { ST_SWAP = 0, ST_TRIAD, ST_SQUEEZE, ST_CONTRACT, ST_RESPLIT, ST_N };

uint32_t stream_id(int step, int kind) { return (uint32_t(step) << 8) | uint32_t(kind); }
constexpr int KIND_SWAP = 0, KIND_TRIAD_A = 1, KIND_TRIAD_X = 2, KIND_TRIAD_Y = 3,
              KIND_TRIAD_D = 4, KIND_SQ_LEFT = 5, KIND_SQ_RIGHT = 8;

GemmDesc G_(const ModeIdx& m, const ModeIdx& n, const ModeIdx& k, double alpha = 1.0,
            double beta = 0.0);
GemmDesc G(const ModeIdx& m, const ModeIdx& n, const ModeIdx& k, double alpha = 1.0,
           double beta = 0.0) {
  GemmDesc g;
  g.m = m;
  g.n = n;
  g.k = k;
  g.alpha = alpha;
  g.beta = beta;
  return g;
}

// Runs [a, b) of consecutive values whose gaps are <= tau times the larger value
// (degenerate multiplets).
std::vector<std::pair<int, int>> multiplets(const std::vector<double>& v, int n, double tau) {
  std::vector<std::pair<int, int>> out;
  int a = 0;
  for (int i = 1; i <= n; ++i) {
    if (i == n || v[i - 1] - v[i] > tau * v[i - 1]) {
      if (i - a > 1) out.push_back({a, i});
      a = i;
    }
  }
  return out;
}

// A truncation to k values never splits a multiplet: move the cut to its first member (or,
// when the multiplet starts at 0, keep it whole).
int64_t multiplet_cut(const std::vector<double>& v, int64_t k, double tau) {
  if (k <= 0 || k >= int64_t(v.size())) return k;
  for (auto& ab : multiplets(v, int(v.size()), tau))
    if (ab.first < k && k < ab.second) return ab.first > 0 ? ab.first : ab.second;
  return k;
}

GemmDesc G_(const ModeIdx& m, const ModeIdx& n, const ModeIdx& k, double alpha, double beta) {
  return G(m, n, k, alpha, beta);
}

int64_t prod(const std::vector<int64_t>& v, size_t a, size_t b) {
  int64_t p = 1;
  for (size_t i = a; i < b && i < v.size(); ++i) p *= v[i];
  return p;
}

}  // namespace

struct tatrg_ctx {
  tatrg_params p;
  cudaStream_t stream;
  Engine eng;
  std::string err;
  // state
  int d = 0;
  std::vector<int64_t> D;  // forward (= backward) leg dims, position 0 = next direction
  int64_t Da = 0;
  DevBuf A, B, sdev;
  std::vector<double> s;
  int step = 0;
  uint32_t replica = 0;     // Philox counter word 2 (sweep index)
  std::vector<double> lnc;  // ln c_k, k = 0..step
  bool ready = false;
  double tau = 1e-10;  // relative gap of a degenerate multiplet (larger in split steps)
  // last step record
  tatrg_step_info info{};
  std::vector<double> spec_s, spec_sigma;
  std::vector<std::vector<double>> spec_sq;
  double flops[ST_N] = {0, 0, 0, 0, 0};
  // Forward-mode tangent along one input (tan_dir 0: beta, 1: h), carried beside the
  // state when tan_on: dA, dB, ds and d ln c_k.  Tangent runs are FP64 throughout.
  bool tan_on = false;
  int tan_dir = 0;
  DevBuf Ad, Bd, sdd;
  std::vector<double> sd, lnc_d;
  double beta0 = 0.0, h0 = 0.0;  // parameters of the last init_ising
  bool ising = false;            // the state comes from init_ising (not set_state)

  tatrg_ctx(const tatrg_params& pp, cudaStream_t s) : p(pp), stream(s), eng(s) {
    eng.stats().timing = pp.profile != 0;
  }
  ~tatrg_ctx() {
    for (cudaStream_t w : side) {
      cudaStreamSynchronize(w);
      cudaStreamDestroy(w);
    }
  }

  // Worker streams for the independent factorisations of one stage, and the launches of
  // the engines that ran on them during the current step.
  std::vector<cudaStream_t> side;
  long side_launches = 0;
  using Task = std::function<void(Engine&)>;
  // Runs the tasks concurrently after the work queued so far on the context's stream, each
  // on its own host thread, stream and engine (the precision of the context's engine); the
  // context's stream then waits for all of them.  A task allocates its outputs on its own
  // stream and rebinds them to the context's stream.  The first error is rethrown.
  void concurrent(std::vector<Task>& tasks);

  int64_t chi() const { return p.chi; }
  int64_t width() const { return int64_t(p.r) * p.chi; }

  double partial_lnz() const {
    // compensated sum of 2^-k ln c_k
    double sum = 0.0, c = 0.0;
    for (size_t k = 0; k < lnc.size(); ++k) {
      double y = std::ldexp(lnc[k], -int(k)) - c;
      double t = sum + y;
      c = (t - sum) - y;
      sum = t;
    }
    return sum;
  }

  void upload_s() {
    sdev = DevBuf(std::max<int64_t>(Da, 1) * sizeof(double), stream);
    TATRG_CUDA(cudaMemcpyAsync(sdev.d(), s.data(), Da * sizeof(double), cudaMemcpyHostToDevice, stream));
    if (tan_on) sdd = eng.upload(sd);
  }
  DevBuf tbuf(int64_t n) { return tan_on ? dalloc(n, stream) : DevBuf(); }

  // Apply the sign convention to the columns of X (F x n, row-major): v = w^T X with the
  // hashed weights; flip the columns (and those of Y, F2 x n, if given) where v < 0.  The
  // tangents Xd, Yd (may be null) flip with them.
  void fix_sign_cols(double* X, int64_t F, int n, double* Y, int64_t F2, double* Xd = nullptr,
                     double* Yd = nullptr) {
    fix_sign_cols_on(stream, X, F, n, Y, F2, Xd, Yd);
  }
  static void fix_sign_cols_on(cudaStream_t st, double* X, int64_t F, int n, double* Y, int64_t F2,
                               double* Xd = nullptr, double* Yd = nullptr) {
    DevBuf v(std::max(n, 1) * sizeof(double), st);
    weighted_colsum(X, F, n, v.d(), st);
    flip_by_sign(X, F, n, nullptr, 0, v.d(), st);
    if (Y) flip_by_sign(Y, F2, n, nullptr, 0, v.d(), st);
    if (Xd) flip_by_sign(Xd, F, n, nullptr, 0, v.d(), st);
    if (Yd) flip_by_sign(Yd, F2, n, nullptr, 0, v.d(), st);
  }
  // Same, but Y is n x F2 (flip its rows).
  void fix_sign_cols_rows(double* X, int64_t F, int n, double* Y, int64_t F2, double* Xd = nullptr,
                          double* Yd = nullptr) {
    DevBuf v(std::max(n, 1) * sizeof(double), stream);
    weighted_colsum(X, F, n, v.d(), stream);
    flip_by_sign(X, F, n, Y, F2, v.d(), stream);
    if (Xd) flip_by_sign(Xd, F, n, Yd, Yd ? F2 : 0, v.d(), stream);
  }

  // Canonical basis of the columns of X (F x n): the sign rule for single columns and, for
  // each degenerate multiplet of vals, the rotation V_M -> V_M O with O the polar factor
  // of V_M^T W (W: hashed weights).  The same rotation is applied to Y: to its rows when
  // y_rows (Y is n x F2), else to its columns (Y is F2 x n).  Xd, Yd: tangents (may be null).
  void canonical_cols(double* X, int64_t F, int n, const std::vector<double>& vals, double* Y,
                      int64_t F2, bool y_rows, double* Xd = nullptr, double* Yd = nullptr);
  void init_ising(double beta, double h, int dd);
  void rg_step();
  void resplit_and_rotate(DMat& phi, DMat& psi, int64_t rows, int64_t Dg,
                          const std::vector<int64_t>& newD, DMat* phid = nullptr,
                          DMat* psid = nullptr);
  double trace();
  double trace_tan(double tt);  // d ln tTr given tTr
  double order_parameter(int leg);
  DMat isometry(Engine& E, const double* rho, int64_t Gd, int kind, std::vector<double>* lam_out,
                const double* rhod = nullptr, DMat* Ud = nullptr);
  void factor(Engine& E, const double* rho, int64_t P, int kind, DMat& Rt, const double* rhod = nullptr,
              DMat* Rtd = nullptr);
};

// ---------------------------------------------------------------------------------
void tatrg_ctx::canonical_cols(double* X, int64_t F, int n, const std::vector<double>& vals,
                               double* Y, int64_t F2, bool y_rows, double* Xd, double* Yd) {
  if (y_rows) fix_sign_cols_rows(X, F, n, Y, F2, Xd, Yd);
  else fix_sign_cols(X, F, n, Y, F2, Xd, Yd);
  const int saved = eng.prec;
  eng.prec = 0;
  for (auto& ab : multiplets(vals, n, tau)) {
    const int a = ab.first, m = ab.second - ab.first;
    TATRG_CHECK(m <= 32, TATRG_ENUMERIC, "degenerate multiplet larger than 32");
    DevBuf G(m * m * sizeof(double), stream), O(m * m * sizeof(double), stream);
    multiplet_overlap(X, F, n, a, m, G.d(), stream);
    SvdResult e = eng.svd(G.d(), m, m);
    eng.mm(m, m, m, e.U.p(), m, false, e.V.p(), m, true, O.d(), m);  // O = U V^T
    DevBuf Od;
    if (Xd) {  // dO from dG = dX_M^T W (the overlap is linear in X)
      DevBuf Gd(m * m * sizeof(double), stream);
      multiplet_overlap(Xd, F, n, a, m, Gd.d(), stream);
      Od = eng.polar_tan(e, Gd.d(), m);
    }
    // X[:, a:a+m] <- X[:, a:a+m] O   (dX_M <- dX_M O + X_M dO, from the old X_M)
    const GemmDesc gx = G_(modes({{F, n, m}}), modes({{m, 1, 1}}), modes({{m, 1, m}}));
    const ModeIdx back = modes({{F, m, n}, {m, 1, 1}});
    DevBuf T(F * m * sizeof(double), stream);
    eng.gemm(gx, X + a, O.d(), T.d());
    if (Xd) {
      DevBuf Td(F * m * sizeof(double), stream);
      eng.gemm(gx, Xd + a, O.d(), Td.d());
      GemmDesc g1 = gx;
      g1.beta = 1.0;
      eng.gemm(g1, X + a, Od.d(), Td.d());
      copy_modes(Xd + a, Td.d(), back, 1.0, stream);
    }
    copy_modes(X + a, T.d(), back, 1.0, stream);
    if (Y) {
      DevBuf T2(F2 * m * sizeof(double), stream);
      if (y_rows) {  // Y[a:a+m, :] <- O^T Y[a:a+m, :]
        const GemmDesc gy = G_(modes({{m, 1, F2}}), modes({{F2, 1, 1}}), modes({{m, m, F2}}));
        eng.gemm(gy, O.d(), Y + a * F2, T2.d());
        if (Yd) {
          DevBuf T2d(F2 * m * sizeof(double), stream);
          eng.gemm(gy, O.d(), Yd + a * F2, T2d.d());
          GemmDesc g1 = gy;
          g1.beta = 1.0;
          eng.gemm(g1, Od.d(), Y + a * F2, T2d.d());
          copy_modes(Yd + a * F2, T2d.d(), modes({{m * F2, 1, 1}}), 1.0, stream);
        }
        copy_modes(Y + a * F2, T2.d(), modes({{m * F2, 1, 1}}), 1.0, stream);
      } else {       // Y[:, a:a+m] <- Y[:, a:a+m] O
        const GemmDesc gy = G_(modes({{F2, n, m}}), modes({{m, 1, 1}}), modes({{m, 1, m}}));
        const ModeIdx backy = modes({{F2, m, n}, {m, 1, 1}});
        eng.gemm(gy, Y + a, O.d(), T2.d());
        if (Yd) {
          DevBuf T2d(F2 * m * sizeof(double), stream);
          eng.gemm(gy, Yd + a, O.d(), T2d.d());
          GemmDesc g1 = gy;
          g1.beta = 1.0;
          eng.gemm(g1, Y + a, Od.d(), T2d.d());
          copy_modes(Yd + a, T2d.d(), backy, 1.0, stream);
        }
        copy_modes(Y + a, T2.d(), backy, 1.0, stream);
      }
    }
  }
  eng.prec = saved;
}

void tatrg_ctx::init_ising(double beta, double h, int dd) {
  d = dd;
  beta0 = beta;
  h0 = h;
  const int64_t n = int64_t(1) << d;
  eng.prec = 0;
  DevBuf T(n * n * sizeof(double), stream);
  ising_tensor(beta, h, d, T.d(), stream);
  SvdResult e = eng.svd(T.d(), n, n);
  double c0 = 0.0;
  for (double x : e.s) c0 += x * x;
  c0 = std::sqrt(c0);
  TATRG_CHECK(c0 > 0.0 && std::isfinite(c0), TATRG_ENUMERIC, "initial tensor has zero norm");
  Da = keep_count(e.s, 1e-14, chi());
  D.assign(d, 2);
  A = DevBuf(n * Da * sizeof(double), stream);
  B = DevBuf(n * Da * sizeof(double), stream);
  copy_modes(A.d(), e.U.p(), modes({{n, e.U.cols, Da}, {Da, 1, 1}}), 1.0, stream);
  copy_modes(B.d(), e.V.p(), modes({{Da, 1, n}, {n, e.V.cols, 1}}), 1.0, stream);
  std::vector<double> ds;
  if (tan_on) {
    DevBuf Td(n * n * sizeof(double), stream);
    ising_tensor_tan(beta, h, d, tan_dir, Td.d(), stream);
    Engine::SvdTan t = eng.svd_tan(Td.d(), n, n, e, int(Da), multiplet_groups(e.s, 1e-10));
    Ad = DevBuf(n * Da * sizeof(double), stream);
    Bd = DevBuf(n * Da * sizeof(double), stream);
    copy_modes(Ad.d(), t.U.p(), modes({{n * Da, 1, 1}}), 1.0, stream);
    copy_modes(Bd.d(), t.V.p(), modes({{Da, 1, n}, {n, Da, 1}}), 1.0, stream);
    ds = t.s;
  }
  fix_sign_cols_rows(A.d(), n, int(Da), B.d(), n, tan_on ? Ad.d() : nullptr, tan_on ? Bd.d() : nullptr);
  s.assign(e.s.begin(), e.s.begin() + Da);
  lnc.assign(1, std::log(c0));
  if (tan_on) {
    // c0 = ||s||, s' = s / c0:  dc0 = s . ds / c0,  ds' = ds / c0 - s dc0 / c0^2
    double dc = 0.0;
    for (int64_t i = 0; i < Da; ++i) dc += s[i] * ds[i];
    dc /= c0;
    sd.assign(Da, 0.0);
    for (int64_t i = 0; i < Da; ++i) sd[i] = ds[i] / c0 - s[i] * dc / (c0 * c0);
    lnc_d.assign(1, dc / c0);
  }
  for (auto& x : s) x /= c0;
  upload_s();
  step = 0;
  ready = true;
  ising = true;
  TATRG_CUDA(cudaStreamSynchronize(stream));
}

double tatrg_ctx::trace() {
  DevBuf out(sizeof(double), stream);
  trace_asb(A.d(), sdev.d(), B.d(), prod(D, 0, D.size()), int(Da), out.d(), stream);
  return eng.to_host(out.d(), 1)[0];
}

// Gu-Wen order parameter X^(m) (Sec. 3): A^(m)[k, l] = sum over the other legs x of
// T[.., x, k, ..; .., x, l, ..] with T = A diag(s) B, the leg at position `leg` open;
// X = (Tr A^(m))^2 / Tr (A^(m))^2.  One FP64 contraction over the traced legs and the bond.
double tatrg_ctx::order_parameter(int leg) {
  const int64_t F = prod(D, 0, D.size()), Dp = D[leg];
  DevBuf As(F * Da * sizeof(double), stream);
  TATRG_CUDA(cudaMemcpyAsync(As.d(), A.d(), As.bytes(), cudaMemcpyDeviceToDevice, stream));
  scale_axis(As.d(), sdev.d(), F, Da, 1, 1, stream);  // A[x, a] s_a
  std::vector<Mode3> kk;
  for (int i = 0; i < d; ++i)
    if (i != leg) kk.push_back({D[i], prod(D, i + 1, d) * Da, prod(D, i + 1, d)});
  kk.push_back({Da, 1, F});
  GemmDesc g;
  g.m = modes({{Dp, prod(D, leg + 1, d) * Da, Dp}});
  g.n = modes({{Dp, prod(D, leg + 1, d), 1}});
  g.k = modes(kk);
  DevBuf Am(Dp * Dp * sizeof(double), stream);
  const int saved = eng.prec;
  eng.prec = 0;
  eng.gemm(g, As.d(), B.d(), Am.d());
  eng.prec = saved;
  const std::vector<double> m = eng.to_host(Am.d(), Dp * Dp);
  double tr = 0.0, tr2 = 0.0;
  for (int64_t i = 0; i < Dp; ++i) {
    tr += m[i * Dp + i];
    for (int64_t j = 0; j < Dp; ++j) tr2 += m[i * Dp + j] * m[j * Dp + i];
  }
  TATRG_CHECK(tr2 != 0.0 && std::isfinite(tr2) && std::isfinite(tr), TATRG_ENUMERIC,
              "order parameter: Tr (A^(m))^2 is zero or not finite");
  return tr * tr / tr2;
}

// d ln tTr = (tTr(dA, s, B) + tTr(A, ds, B) + tTr(A, s, dB)) / tTr
double tatrg_ctx::trace_tan(double tt) {
  const int64_t F = prod(D, 0, D.size());
  DevBuf out(3 * sizeof(double), stream);
  trace_asb(Ad.d(), sdev.d(), B.d(), F, int(Da), out.d(), stream);
  trace_asb(A.d(), sdd.d(), B.d(), F, int(Da), out.d() + 1, stream);
  trace_asb(A.d(), sdev.d(), Bd.d(), F, int(Da), out.d() + 2, stream);
  std::vector<double> v = eng.to_host(out.d(), 3);
  return (v[0] + v[1] + v[2]) / tt;
}

// Leading eigenvectors of a PSD Gram (Eqs. 2-3): exact (k >= G) or RSVD with ell = k.
// With rhod (tangent mode) also the tangent of U in *Ud (constant for ATRG).
DMat tatrg_ctx::isometry(Engine& E, const double* rho, int64_t Gd, int kind, std::vector<double>* lam_out,
                         const double* rhod, DMat* Ud) {
  cudaStream_t stream = E.stream();
  DMat U;
  if (p.method == TATRG_ATRG) {
    U.buf = dalloc(Gd * Gd, stream);
    U.rows = U.cols = Gd;
    fill(U.p(), Gd * Gd, 0.0, stream);
    ModeIdx diag = modes({{Gd, 0, Gd + 1}});
    DevBuf one(sizeof(double), stream);
    fill(one.d(), 1, 1.0, stream);
    copy_modes(U.p(), one.d(), diag, 1.0, stream);
    if (rhod && Ud) {
      Ud->buf = dalloc(Gd * Gd, stream);
      Ud->rows = Ud->cols = Gd;
      fill(Ud->p(), Gd * Gd, 0.0, stream);
    }
    return U;
  }
  const int64_t k = std::min(width(), Gd);
  SvdResult e;
  Engine::SvdTan et;
  if (k >= Gd) {
    e = E.svd(rho, Gd, Gd);
    if (rhod) et = E.svd_tan(rhod, Gd, Gd, e, keep_count(e.s, 1e-14, k), multiplet_groups(e.s, tau));
  } else {
    DevBuf om(Gd * k * sizeof(double), stream);
    gaussian(p.seed, stream_id(step, kind), replica, Gd * k, om.d(), stream, !E.fp64_grade());
    if (rhod) {
      Engine::RsvdT r = E.rsvd_psd_t(rho, rhod, Gd, k, p.q, om.d(), tau);
      e = std::move(r.e);
      et = std::move(r.t);
    } else {
      e = E.rsvd_psd(rho, Gd, k, p.q, om.d());
    }
  }
  int keep = keep_count(e.s, 1e-14, k);
  TATRG_CHECK(keep >= 1, TATRG_ENUMERIC, "triad Gram is zero");
  U.buf = dalloc(Gd * keep, stream);
  U.rows = Gd;
  U.cols = keep;
  copy_modes(U.p(), e.U.p(), modes({{Gd, e.U.cols, keep}, {keep, 1, 1}}), 1.0, stream);
  if (rhod) {
    Ud->buf = dalloc(Gd * keep, stream);
    Ud->rows = Gd;
    Ud->cols = keep;
    copy_modes(Ud->p(), et.U.p(), modes({{Gd, et.U.cols, keep}, {keep, 1, 1}}), 1.0, stream);
  }
  fix_sign_cols_on(stream, U.p(), Gd, keep, nullptr, 0, rhod ? Ud->p() : nullptr);
  if (lam_out) *lam_out = e.s;
  return U;
}

// rho ~= R^T R from the leading eigenpairs (exact when ell >= P); returns R^T (P x keep),
// and with rhod its tangent in *Rtd: d(U sqrt(l)) = dU sqrt(l) + U dl / (2 sqrt(l)).
void tatrg_ctx::factor(Engine& E, const double* rho, int64_t P, int kind, DMat& Rt, const double* rhod,
                       DMat* Rtd) {
  cudaStream_t stream = E.stream();
  const int64_t ell = std::min(width(), P);
  SvdResult e;
  Engine::SvdTan et;
  if (ell >= P) {
    e = E.svd(rho, P, P);
    if (rhod) et = E.svd_tan(rhod, P, P, e, keep_count(e.s, 1e-14, ell), multiplet_groups(e.s, tau));
  } else {
    DevBuf om(P * ell * sizeof(double), stream);
    gaussian(p.seed, stream_id(step, kind), replica, P * ell, om.d(), stream, !E.fp64_grade());
    if (rhod) {
      Engine::RsvdT r = E.rsvd_psd_t(rho, rhod, P, ell, p.q, om.d(), tau);
      e = std::move(r.e);
      et = std::move(r.t);
    } else {
      e = E.rsvd_psd(rho, P, ell, p.q, om.d());
    }
  }
  int keep = keep_count(e.s, 1e-14, ell);
  TATRG_CHECK(keep >= 1, TATRG_ENUMERIC, "squeezer Gram is zero");
  Rt.buf = dalloc(P * keep, stream);
  Rt.rows = P;
  Rt.cols = keep;
  copy_modes(Rt.p(), e.U.p(), modes({{P, e.U.cols, keep}, {keep, 1, 1}}), 1.0, stream);
  std::vector<double> sq(e.s.begin(), e.s.begin() + keep);
  for (auto& x : sq) x = std::sqrt(std::max(x, 0.0));
  DevBuf sqd(keep * sizeof(double), stream);
  TATRG_CUDA(cudaMemcpyAsync(sqd.d(), sq.data(), keep * sizeof(double), cudaMemcpyHostToDevice, stream));
  if (rhod) {
    std::vector<double> dsq(keep);
    for (int i = 0; i < keep; ++i) dsq[i] = et.s[i] / (2.0 * sq[i]);
    DevBuf dsqd = E.upload(dsq);
    Rtd->buf = dalloc(P * keep, stream);
    Rtd->rows = P;
    Rtd->cols = keep;
    copy_modes(Rtd->p(), et.U.p(), modes({{P, et.U.cols, keep}, {keep, 1, 1}}), 1.0, stream);
    scale_axis_tan(Rt.p(), Rtd->p(), sqd.d(), dsqd.d(), P, keep, 1, 1, stream);
  } else {
    scale_axis(Rt.p(), sqd.d(), P, keep, 1, 1, stream);
  }
  TATRG_CUDA(cudaStreamSynchronize(stream));
}

void tatrg_ctx::concurrent(std::vector<Task>& tasks) {
  const size_t n = tasks.size();
  while (side.size() < n) {
    cudaStream_t w;
    TATRG_CUDA(cudaStreamCreateWithFlags(&w, cudaStreamNonBlocking));
    side.push_back(w);
  }
  cudaEvent_t ready;
  TATRG_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
  TATRG_CUDA(cudaEventRecord(ready, stream));
  std::vector<std::exception_ptr> err(n);
  std::vector<std::unique_ptr<Engine>> engines(n);
  std::vector<std::thread> threads;
  auto work = [&](size_t i) {
    try {
      TATRG_CUDA(cudaStreamWaitEvent(side[i], ready, 0));
      engines[i] = std::make_unique<Engine>(side[i]);
      Engine& e = *engines[i];
      e.prec = eng.prec;
      e.allow_tc = eng.allow_tc;
      e.stats().timing = eng.stats().timing;
      tasks[i](e);
    } catch (...) {
      err[i] = std::current_exception();
    }
  };
  for (size_t i = 0; i < n; ++i) {
    try {
      threads.emplace_back(work, i);
    } catch (...) {  // no thread: run the task here
      work(i);
    }
  }
  for (auto& t : threads) t.join();
  for (size_t i = 0; i < n; ++i) {
    cudaEvent_t done;
    TATRG_CUDA(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
    TATRG_CUDA(cudaEventRecord(done, side[i]));
    TATRG_CUDA(cudaStreamWaitEvent(stream, done, 0));
    TATRG_CUDA(cudaEventDestroy(done));
    if (engines[i]) side_launches += engines[i]->stats().launches;
  }
  TATRG_CUDA(cudaEventDestroy(ready));
  for (auto& e : err)
    if (e) std::rethrow_exception(e);
}

namespace {
struct StageTimer {
  cudaEvent_t ev[ST_N + 1];
  cudaStream_t s;
  explicit StageTimer(cudaStream_t st) : s(st) {
    for (auto& e : ev) cudaEventCreate(&e);
  }
  ~StageTimer() {
    for (auto& e : ev) cudaEventDestroy(e);
  }
  void mark(int i) { cudaEventRecord(ev[i], s); }
};
}  // namespace

void tatrg_ctx::rg_step() {
  TATRG_CHECK(ready, TATRG_ESTATE, "rg_step before init_ising / set_state");
  step++;
  const bool split = p.precision != TATRG_FP64 && step >= std::max(1, p.split_from_step);
  const int mask = p.split_stages ? p.split_stages : 31;
  // precision schedule: FP64 before split_from_step, early_precision until late_from_step
  const int prec_now = (p.early_precision != 0 && step < p.late_from_step) ? p.early_precision : p.precision;
  // multiplet gap: above the rounding of the float-grade forms, the oracle's 1e-10 otherwise
  tau = (split && prec_now != TATRG_OZAKI) ? 1e-6 : 1e-10;
  auto stage_prec = [&](Stage sg) { eng.prec = (split && (mask >> sg) & 1) ? prec_now : 0; };
  stage_prec(ST_SWAP);
  cudaStream_t st = stream;
  StageTimer tm(st);
  const long launches0 = eng.stats().launches, tc0 = eng.stats().tc_launches;
  const double tcf0 = eng.stats().flops_tc;
  eng.stats().drain_ms();
  side_launches = 0;
  for (auto& f : flops) f = 0.0;
  auto count = [&](Stage sg, const GemmDesc& g) {
    flops[sg] += 2.0 * double(g.m.total()) * double(g.n.total()) * double(g.k.total());
  };
  auto run = [&](Stage sg, const GemmDesc& g, const double* a, const double* b, double* c) {
    count(sg, g);
    eng.gemm(g, a, b, c);
  };
  // Tangent mode: every bilinear contraction c = g(a, b) also gives dc = g(da, b) + g(a, db);
  // a null tangent is a constant operand.
  const bool T = tan_on;
  TATRG_CHECK(!T || !split, TATRG_EINVAL, "tangent runs are FP64");
  auto run2 = [&](Stage sg, const GemmDesc& g, const double* a, const double* da, const double* b,
                  const double* db, double* c, double* dc) {
    run(sg, g, a, b, c);
    if (!T) return;
    GemmDesc g2 = g;
    g2.beta = 0.0;
    if (da) {
      eng.gemm(g2, da, b, dc);
      g2.beta = 1.0;
    }
    if (db) {
      eng.gemm(g2, a, db, dc);
      g2.beta = 1.0;
    }
    TATRG_CHECK(g2.beta == 1.0, TATRG_EINVAL, "tangent contraction without a tangent operand");
  };
  auto tp = [&](const DevBuf& b) -> double* { return T ? b.d() : nullptr; };
  auto tpm = [&](const DMat& b) -> double* { return T ? b.p() : nullptr; };

  const int g = d - 2;
  const int64_t D0 = D[0];
  const int64_t I = prod(D, 1, d);
  const int64_t Gd = g > 0 ? prod(D, 1, 1 + g) : 1;
  const int64_t Ds = D[d - 1];
  const int64_t Da_ = Da;

  // ============================ bond swap (Eq. 1) ============================
  tm.mark(0);
  DevBuf As(D0 * I * Da_ * sizeof(double), st), Bs(Da_ * D0 * I * sizeof(double), st);
  TATRG_CUDA(cudaMemcpyAsync(As.d(), A.d(), As.bytes(), cudaMemcpyDeviceToDevice, st));
  TATRG_CUDA(cudaMemcpyAsync(Bs.d(), B.d(), Bs.bytes(), cudaMemcpyDeviceToDevice, st));
  DevBuf Asd = tbuf(D0 * I * Da_), Bsd = tbuf(Da_ * D0 * I);
  if (T) {
    TATRG_CUDA(cudaMemcpyAsync(Asd.d(), Ad.d(), As.bytes(), cudaMemcpyDeviceToDevice, st));
    TATRG_CUDA(cudaMemcpyAsync(Bsd.d(), Bd.d(), Bs.bytes(), cudaMemcpyDeviceToDevice, st));
    scale_axis_tan(As.d(), Asd.d(), sdev.d(), sdd.d(), D0 * I, Da_, 1, 1, st);
    scale_axis_tan(Bs.d(), Bsd.d(), sdev.d(), sdd.d(), 1, Da_, D0 * I, 1, st);
  } else {
    scale_axis(As.d(), sdev.d(), D0 * I, Da_, 1, 1, st);  // A[k,i,b] s_b
    scale_axis(Bs.d(), sdev.d(), 1, Da_, D0 * I, 1, st);  // s_a B[a,k,j]
  }
  const int64_t rows = Da_ * I;
  const int64_t ell = std::min(width(), rows);
  SvdResult sw;
  Engine::SvdTan swt;  // tangent mode: tangents of the leading singular triplets
  info.swap_exact = 0;
  if (ell >= rows) {
    // dense Mid[(a,i),(b,j)] = sum_k Bs[a,k,j] As[k,i,b], one contraction per (a, b)
    info.swap_exact = 1;
    DevBuf mid(rows * rows * sizeof(double), st), midd = tbuf(rows * rows);
    for (int64_t a = 0; a < Da_; ++a)
      for (int64_t b = 0; b < Da_; ++b) {
        GemmDesc gm = G(modes({{I, Da_, rows}}), modes({{I, 1, 1}}), modes({{D0, I * Da_, I}}));
        const int64_t oa = b, ob = a * D0 * I, oc = a * I * rows + b * I;
        run2(ST_SWAP, gm, As.d() + oa, T ? Asd.d() + oa : nullptr, Bs.d() + ob, T ? Bsd.d() + ob : nullptr,
             mid.d() + oc, T ? midd.d() + oc : nullptr);
      }
    sw = eng.svd(mid.d(), rows, rows);
    if (T) swt = eng.svd_tan(midd.d(), rows, rows, sw, keep_count(sw.s, 1e-14, sw.r), multiplet_groups(sw.s, tau));
  } else {
    // the swap sketch Omega (rows x ell), stored only when a product needs it from memory
    DevBuf om;
    const GaussSrc swap_sketch{p.seed, stream_id(step, KIND_SWAP), replica};
    auto materialise = [&]() {
      if (!om.empty()) return;
      om = DevBuf(rows * ell * sizeof(double), st);
      gaussian(swap_sketch.seed, swap_sketch.sid, swap_sketch.replica, rows * ell, om.d(), st, !eng.fp64_grade());
    };
    // M X: W[a,k,b,p] = sum_j Bs[a,k,j] X[(b,j),p];  Y[(a,i),p] = sum_{k,b} As[k,i,b] W[a,k,b,p]
    // (with any pair of factors Ap, Bp in place of As, Bs; beta = 1 accumulates into Y)
    auto apply_g = [&](const double* Ap, const double* Bp, const double* X, int64_t w, double* Y,
                       double beta) {
      DevBuf W(Da_ * D0 * Da_ * w * sizeof(double), st);
      run(ST_SWAP,
          G(modes({{Da_ * D0, I, Da_ * w}}), modes({{Da_, I * w, w}, {w, 1, 1}}), modes({{I, 1, w}})),
          Bp, X, W.d());
      run(ST_SWAP,
          G(modes({{I, Da_, w}}), modes({{Da_, D0 * Da_ * w, I * w}, {w, 1, 1}}),
            modes({{D0, I * Da_, Da_ * w}, {Da_, 1, w}}), 1.0, beta),
          Ap, W.d(), Y);
    };
    // M^T X: W[a,k,b,p] = sum_i As[k,i,b] X[(a,i),p];  Z[(b,j),p] = sum_{a,k} Bs[a,k,j] W[a,k,b,p]
    auto rapply_g = [&](const double* Ap, const double* Bp, const double* X, int64_t w, double* Z,
                        double beta) {
      DevBuf W(Da_ * D0 * Da_ * w * sizeof(double), st);
      run(ST_SWAP,
          G(modes({{D0, I * Da_, Da_ * w}, {Da_, 1, w}}), modes({{Da_, I * w, D0 * Da_ * w}, {w, 1, 1}}),
            modes({{I, Da_, w}})),
          Ap, X, W.d());
      run(ST_SWAP,
          G(modes({{I, 1, w}}), modes({{Da_, w, I * w}, {w, 1, 1}}), modes({{Da_ * D0, I, Da_ * w}}), 1.0,
            beta),
          Bp, W.d(), Z);
    };
    auto apply = [&](const double* X, int64_t w, double* Y) { apply_g(As.d(), Bs.d(), X, w, Y, 0.0); };
    auto rapply = [&](const double* X, int64_t w, double* Z) { rapply_g(As.d(), Bs.d(), X, w, Z, 0.0); };
    // dM X = dAs-part + dBs-part (Mid is bilinear in As, Bs)
    auto apply_d = [&](const double* X, int64_t w, double* Y) {
      apply_g(Asd.d(), Bs.d(), X, w, Y, 0.0);
      apply_g(As.d(), Bsd.d(), X, w, Y, 1.0);
    };
    auto rapply_d = [&](const double* X, int64_t w, double* Z) {
      rapply_g(Asd.d(), Bs.d(), X, w, Z, 0.0);
      rapply_g(As.d(), Bsd.d(), X, w, Z, 1.0);
    };
    // Compressed randomized SVD.  Mid = L R with the inner index (a, k, b):
    //   (R x)[a,k,b] = sum_j Bs[a,k,j] x[(b,j)],  (L w)[(a,i)] = sum_{k,b} As[k,i,b] w[a,k,b];
    // every basis of the subspace iteration lies in range(L) or range(R^T), so it is kept
    // as Q = L V (or R^T V) and orthonormalised in the metrics L^T L = 1 (x) G_A and
    // R R^T = G_B (x) 1, with G_A[(k,b),(k',b')] = sum_i As As and
    // G_B[(a,k),(a',k')] = sum_j Bs Bs.  Same subspaces as the explicit iteration, without
    // the rows x ell panels; only X and Y are formed at the end.
    const int64_t nin = D0 * Da_;
    const int64_t nL = Da_ * nin;  // rows of an inner panel [a][k][b]
    bool done = false;
    if (nL > ell && !T) {  // tangent runs take the explicit iteration (the same subspaces)
      DevBuf GA(nin * nin * sizeof(double), st), GB(nin * nin * sizeof(double), st);
      run(ST_SWAP,
          G(modes({{D0, I * Da_, Da_ * nin}, {Da_, 1, nin}}), modes({{D0, I * Da_, Da_}, {Da_, 1, 1}}),
            modes({{I, Da_, Da_}})),
          As.d(), As.d(), GA.d());
      run(ST_SWAP, G(modes({{nin, I, nin}}), modes({{nin, I, 1}}), modes({{I, 1, 1}})), Bs.d(), Bs.d(), GB.d());
      auto metric_L = [&](const double* V, int64_t w, double* U) {  // (1 (x) G_A) V
        run(ST_SWAP,
            G(modes({{nin, nin, w}}), modes({{Da_, nin * w, nin * w}, {w, 1, 1}}), modes({{nin, 1, w}})),
            GA.d(), V, U);
      };
      auto metric_R = [&](const double* V, int64_t w, double* U) {  // (G_B (x) 1) V
        run(ST_SWAP, G(modes({{nin, nin, Da_ * w}}), modes({{Da_ * w, 1, 1}}), modes({{nin, 1, Da_ * w}})),
            GB.d(), V, U);
      };
      auto apply_R = [&](const double* X, int64_t w, double* W) {  // W = R X
        run(ST_SWAP,
            G(modes({{Da_ * D0, I, Da_ * w}}), modes({{Da_, I * w, w}, {w, 1, 1}}), modes({{I, 1, w}})),
            Bs.d(), X, W);
      };
      auto apply_L = [&](const double* W, int64_t w, double* Y) {  // Y = L W
        run(ST_SWAP,
            G(modes({{I, Da_, w}}), modes({{Da_, D0 * Da_ * w, I * w}, {w, 1, 1}}),
              modes({{D0, I * Da_, Da_ * w}, {Da_, 1, w}})),
            As.d(), W, Y);
      };
      auto apply_Rt = [&](const double* W, int64_t w, double* Z) {  // Z = R^T W
        run(ST_SWAP,
            G(modes({{I, 1, w}}), modes({{Da_, w, I * w}, {w, 1, 1}}), modes({{Da_ * D0, I, Da_ * w}})),
            Bs.d(), W, Z);
      };
      DMat W0;
      W0.buf = dalloc(nL * ell, st);
      {
        // W0 = R Omega; in split precision the sketch is generated in the operand packer
        const GemmDesc gr = G(modes({{Da_ * D0, I, Da_ * ell}}), modes({{Da_, I * ell, ell}, {ell, 1, 1}}),
                              modes({{I, 1, ell}}));
        if (eng.gemm_gauss_b(gr, Bs.d(), swap_sketch, W0.p())) {
          count(ST_SWAP, gr);
        } else {
          materialise();
          apply_R(om.d(), ell, W0.p());
        }
      }
      om.release();
      Engine::MetricOrth Qm = eng.orth_metric(W0.p(), nL, ell, metric_L);
      bool ok = Qm.ok;
      for (int it = 0; ok && it < p.q; ++it) {
        Engine::MetricOrth Qt = eng.orth_metric(Qm.U.p(), nL, ell, metric_R);
        ok = Qt.ok;
        if (ok) {
          Qm = eng.orth_metric(Qt.U.p(), nL, ell, metric_L);
          ok = Qm.ok;
        }
      }
      Engine::MetricOrth Pm;
      if (ok) {
        Pm = eng.orth_metric(Qm.U.p(), nL, ell, metric_R);  // B^T = R^T U = P R
        ok = Pm.ok;
      }
      if (ok) {
        DevBuf Rt(ell * ell * sizeof(double), st);
        transpose(Pm.R.p(), ell, ell, Rt.d(), st);
        SvdResult c = eng.svd(Rt.d(), ell, ell);  // R^T = W S Z^T
        const int64_t r = c.r;
        // explicit singular vectors: U = L (V W), V = R^T (V_P Z)
        DMat WX, WY;
        WX.buf = dalloc(nL * r, st);
        WY.buf = dalloc(nL * r, st);
        eng.mm(nL, r, ell, Qm.V.p(), ell, false, c.U.p(), c.U.cols, false, WX.p(), r);
        eng.mm(nL, r, ell, Pm.V.p(), ell, false, c.V.p(), c.V.cols, false, WY.p(), r);
        sw.r = int(r);
        sw.s = c.s;
        sw.S = std::move(c.S);
        sw.U.buf = dalloc(rows * r, st);
        sw.U.rows = rows;
        sw.U.cols = r;
        sw.V.buf = dalloc(rows * r, st);
        sw.V.rows = rows;
        sw.V.cols = r;
        apply_L(WX.p(), r, sw.U.p());
        apply_Rt(WY.p(), r, sw.V.p());
        done = true;
      }
    }
    if (!done) {
      materialise();
      if (T) {
        Engine::RsvdT r = eng.rsvd_t(apply, rapply, apply_d, rapply_d, rows, rows, ell, p.q, om.d(), tau);
        sw = std::move(r.e);
        swt = std::move(r.t);
      } else {
        sw = eng.rsvd(apply, rapply, rows, rows, ell, p.q, om.d());
      }
    }
  }
  const int64_t Dg = multiplet_cut(sw.s, keep_count(sw.s, 1e-14, chi()), tau);
  TATRG_CHECK(Dg >= 1, TATRG_ENUMERIC, "bond swap: zero middle tensor");
  info.swap_gap = (Dg < int64_t(sw.s.size())) ? (sw.s[Dg - 1] - sw.s[Dg]) / sw.s[0] : INFINITY;
  spec_sigma = sw.s;
  // X[(a,i),g], Y[(b,j),g] with the sign convention on X
  DevBuf X(rows * Dg * sizeof(double), st), Y(rows * Dg * sizeof(double), st);
  copy_modes(X.d(), sw.U.p(), modes({{rows, sw.U.cols, Dg}, {Dg, 1, 1}}), 1.0, st);
  copy_modes(Y.d(), sw.V.p(), modes({{rows, sw.V.cols, Dg}, {Dg, 1, 1}}), 1.0, st);
  DevBuf Xd = tbuf(rows * Dg), Yd = tbuf(rows * Dg), sigdd;
  if (T) {
    TATRG_CHECK(swt.U.cols >= Dg, TATRG_ENUMERIC, "bond swap: tangent of a cut below the rounding floor");
    copy_modes(Xd.d(), swt.U.p(), modes({{rows, swt.U.cols, Dg}, {Dg, 1, 1}}), 1.0, st);
    copy_modes(Yd.d(), swt.V.p(), modes({{rows, swt.V.cols, Dg}, {Dg, 1, 1}}), 1.0, st);
    sigdd = eng.upload(std::vector<double>(swt.s.begin(), swt.s.begin() + Dg));
  }
  fix_sign_cols(X.d(), rows, int(Dg), Y.d(), rows, tp(Xd), tp(Yd));
  std::vector<double> sig(sw.s.begin(), sw.s.begin() + Dg);
  DevBuf sigd(Dg * sizeof(double), st);
  TATRG_CUDA(cudaMemcpyAsync(sigd.d(), sig.data(), Dg * sizeof(double), cudaMemcpyHostToDevice, st));
  As.release();
  Bs.release();
  Asd.release();
  Bsd.release();

  // ======================== triad isometries and tensors (Eqs. 2-4) ========================
  tm.mark(1);
  stage_prec(ST_TRIAD);
  const int64_t nx = Da_ * Gd * Ds * Dg;  // elements of X (= Y)
  DevBuf Xs(nx * sizeof(double), st), Ys(nx * sizeof(double), st);
  TATRG_CUDA(cudaMemcpyAsync(Xs.d(), X.d(), nx * sizeof(double), cudaMemcpyDeviceToDevice, st));
  TATRG_CUDA(cudaMemcpyAsync(Ys.d(), Y.d(), nx * sizeof(double), cudaMemcpyDeviceToDevice, st));
  DevBuf Xsd = tbuf(nx), Ysd = tbuf(nx);
  if (T) {
    TATRG_CUDA(cudaMemcpyAsync(Xsd.d(), Xd.d(), nx * sizeof(double), cudaMemcpyDeviceToDevice, st));
    TATRG_CUDA(cudaMemcpyAsync(Ysd.d(), Yd.d(), nx * sizeof(double), cudaMemcpyDeviceToDevice, st));
    scale_axis_tan(Xs.d(), Xsd.d(), sigd.d(), sigdd.d(), Da_ * Gd * Ds, Dg, 1, 2, st);
    scale_axis_tan(Ys.d(), Ysd.d(), sigd.d(), sigdd.d(), Da_ * Gd * Ds, Dg, 1, 2, st);
  } else {
    scale_axis(Xs.d(), sigd.d(), Da_ * Gd * Ds, Dg, 1, 2, st);
    scale_axis(Ys.d(), sigd.d(), Da_ * Gd * Ds, Dg, 1, 2, st);
  }
  const int64_t GSg = Gd * Ds * Dg;
  DevBuf xi_x(Da_ * Da_ * sizeof(double), st), xi_y(Da_ * Da_ * sizeof(double), st);
  DevBuf xi_xd = tbuf(Da_ * Da_), xi_yd = tbuf(Da_ * Da_);
  run2(ST_TRIAD, G(modes({{Da_, GSg, Da_}}), modes({{Da_, GSg, 1}}), modes({{GSg, 1, 1}})), Xs.d(), tp(Xsd),
       X.d(), tp(Xd), xi_x.d(), tp(xi_xd));
  run2(ST_TRIAD, G(modes({{Da_, GSg, Da_}}), modes({{Da_, GSg, 1}}), modes({{GSg, 1, 1}})), Ys.d(), tp(Ysd),
       Y.d(), tp(Yd), xi_y.d(), tp(xi_yd));
  DevBuf rho_a(Gd * Gd * sizeof(double), st), rho_x(Gd * Gd * sizeof(double), st),
      rho_y(Gd * Gd * sizeof(double), st), rho_d(Gd * Gd * sizeof(double), st);
  DevBuf rho_ad = tbuf(Gd * Gd), rho_xd = tbuf(Gd * Gd), rho_yd = tbuf(Gd * Gd), rho_dd = tbuf(Gd * Gd);
  {
    // t_a[i0,G,s,a'] = sum_a A[i0,G,s,a] Xi_X[a,a'];  rho_A[G,G'] = sum t_a[i0,G,s,a] A[i0,G',s,a]
    DevBuf ta(D0 * Gd * Ds * Da_ * sizeof(double), st), tad = tbuf(D0 * Gd * Ds * Da_);
    run2(ST_TRIAD, G(modes({{D0 * Gd * Ds, Da_, Da_}}), modes({{Da_, 1, 1}}), modes({{Da_, 1, Da_}})),
         A.d(), tp(Ad), xi_x.d(), tp(xi_xd), ta.d(), tp(tad));
    run2(ST_TRIAD,
         G(modes({{Gd, Ds * Da_, Gd}}), modes({{Gd, Ds * Da_, 1}}),
           modes({{D0, Gd * Ds * Da_, Gd * Ds * Da_}, {Ds * Da_, 1, 1}})),
         ta.d(), tp(tad), A.d(), tp(Ad), rho_a.d(), tp(rho_ad));
    // rho_X[G,G'] = sum_{a,s,g} Xs[a,G,s,g] X[a,G',s,g]  (and rho_Y)
    GemmDesc gx = G(modes({{Gd, Ds * Dg, Gd}}), modes({{Gd, Ds * Dg, 1}}),
                    modes({{Da_, GSg, GSg}, {Ds * Dg, 1, 1}}));
    run2(ST_TRIAD, gx, Xs.d(), tp(Xsd), X.d(), tp(Xd), rho_x.d(), tp(rho_xd));
    run2(ST_TRIAD, gx, Ys.d(), tp(Ysd), Y.d(), tp(Yd), rho_y.d(), tp(rho_yd));
    // t_d[b',j0,G,s] = sum_b Xi_Y[b,b'] D[b,j0,G,s];  rho_D = sum t_d[b,j0,G,s] D[b,j0,G',s]
    DevBuf td(Da_ * D0 * Gd * Ds * sizeof(double), st), tdd = tbuf(Da_ * D0 * Gd * Ds);
    const int64_t JGS = D0 * Gd * Ds;
    run2(ST_TRIAD, G(modes({{Da_, 1, JGS}}), modes({{JGS, 1, 1}}), modes({{Da_, Da_, JGS}})),
         xi_y.d(), tp(xi_yd), B.d(), tp(Bd), td.d(), tp(tdd));
    run2(ST_TRIAD,
         G(modes({{Gd, Ds, Gd}}), modes({{Gd, Ds, 1}}), modes({{Da_ * D0, Gd * Ds, Gd * Ds}, {Ds, 1, 1}})),
         td.d(), tp(tdd), B.d(), tp(Bd), rho_d.d(), tp(rho_dd));
  }
  Xs.release();
  Ys.release();
  Xsd.release();
  Ysd.release();
  DMat UAd, UXd, UYd, UDd;
  DMat UA, UX, UY, UD;
  if (!T) {
    // the four isometries are independent: factorise the Grams concurrently
    std::vector<Task> tasks;
    const double* rhos[4] = {rho_a.d(), rho_x.d(), rho_y.d(), rho_d.d()};
    DMat* outs[4] = {&UA, &UX, &UY, &UD};
    const int kinds[4] = {KIND_TRIAD_A, KIND_TRIAD_X, KIND_TRIAD_Y, KIND_TRIAD_D};
    for (int i = 0; i < 4; ++i)
      tasks.push_back([&, i](Engine& E) {
        *outs[i] = isometry(E, rhos[i], Gd, kinds[i], nullptr);
        outs[i]->buf.rebind(st);
      });
    concurrent(tasks);
  } else {
    UA = isometry(eng, rho_a.d(), Gd, KIND_TRIAD_A, nullptr, tp(rho_ad), &UAd);
    UX = isometry(eng, rho_x.d(), Gd, KIND_TRIAD_X, nullptr, tp(rho_xd), &UXd);
    UY = isometry(eng, rho_y.d(), Gd, KIND_TRIAD_Y, nullptr, tp(rho_yd), &UYd);
    UD = isometry(eng, rho_d.d(), Gd, KIND_TRIAD_D, nullptr, tp(rho_dd), &UDd);
  }
  const int64_t KA = UA.cols, KX = UX.cols, KY = UY.cols, KD = UD.cols;
  // E[i0,kA,s,a] = sum_G A[i0,G,s,a] UA[G,kA]
  DevBuf E(D0 * KA * Ds * Da_ * sizeof(double), st), F(Da_ * KX * Ds * Dg * sizeof(double), st),
      Gt(Da_ * KY * Ds * Dg * sizeof(double), st), H(D0 * KD * Ds * Da_ * sizeof(double), st);
  DevBuf Ed = tbuf(D0 * KA * Ds * Da_), Fd = tbuf(Da_ * KX * Ds * Dg), Gtd = tbuf(Da_ * KY * Ds * Dg),
         Hd = tbuf(D0 * KD * Ds * Da_);
  run2(ST_TRIAD,
       G(modes({{D0, Gd * Ds * Da_, KA * Ds * Da_}, {Ds * Da_, 1, 1}}), modes({{KA, 1, Ds * Da_}}),
         modes({{Gd, Ds * Da_, KA}})),
       A.d(), tp(Ad), UA.p(), tpm(UAd), E.d(), tp(Ed));
  // F[a,kX,s,g] = sum_G X[a,G,s,g] UX[G,kX] sigma_g ;  G[b,kY,s,g] likewise with Y
  run2(ST_TRIAD,
       G(modes({{Da_, GSg, KX * Ds * Dg}, {Ds * Dg, 1, 1}}), modes({{KX, 1, Ds * Dg}}),
         modes({{Gd, Ds * Dg, KX}})),
       X.d(), tp(Xd), UX.p(), tpm(UXd), F.d(), tp(Fd));
  if (T) scale_axis_tan(F.d(), Fd.d(), sigd.d(), sigdd.d(), Da_ * KX * Ds, Dg, 1, 1, st);
  else scale_axis(F.d(), sigd.d(), Da_ * KX * Ds, Dg, 1, 1, st);
  run2(ST_TRIAD,
       G(modes({{Da_, GSg, KY * Ds * Dg}, {Ds * Dg, 1, 1}}), modes({{KY, 1, Ds * Dg}}),
         modes({{Gd, Ds * Dg, KY}})),
       Y.d(), tp(Yd), UY.p(), tpm(UYd), Gt.d(), tp(Gtd));
  // H[j0,kD,s,b] = sum_G D[b,j0,G,s] UD[G,kD]
  run2(ST_TRIAD,
       G(modes({{D0, Gd * Ds, KD * Ds * Da_}, {Ds, 1, Da_}, {Da_, D0 * Gd * Ds, 1}}),
         modes({{KD, 1, Ds * Da_}}), modes({{Gd, Ds, KD}})),
       B.d(), tp(Bd), UD.p(), tpm(UDd), H.d(), tp(Hd));
  X.release();
  Y.release();
  Xd.release();
  Yd.release();

  // ============================ squeezers (Eq. 5) ============================
  tm.mark(2);
  stage_prec(ST_SQUEEZE);
  std::vector<DMat> Ms(d - 1), Nts(d - 1);  // M[(a,b),k] and N^T[(a,b),k]
  std::vector<DMat> Msd(d - 1), Ntsd(d - 1);  // their tangents (tangent mode)
  std::vector<int64_t> Kn(d - 1, 0);
  spec_sq.assign(d - 1, {});
  {
    DevBuf om_d(Da_ * Da_ * sizeof(double), st), om_y(Dg * Dg * sizeof(double), st),
        om_a(Da_ * Da_ * sizeof(double), st), om_x(Dg * Dg * sizeof(double), st);
    DevBuf om_dd = tbuf(Da_ * Da_), om_yd = tbuf(Dg * Dg), om_ad = tbuf(Da_ * Da_), om_xd = tbuf(Dg * Dg);
    const int64_t JKS = D0 * KD * Ds, IKS = D0 * KA * Ds;
    run2(ST_SQUEEZE, G(modes({{Da_, 1, Da_}}), modes({{Da_, 1, 1}}), modes({{JKS, Da_, Da_}})), H.d(), tp(Hd),
         H.d(), tp(Hd), om_d.d(), tp(om_dd));
    run2(ST_SQUEEZE, G(modes({{Da_, 1, Da_}}), modes({{Da_, 1, 1}}), modes({{IKS, Da_, Da_}})), E.d(), tp(Ed),
         E.d(), tp(Ed), om_a.d(), tp(om_ad));
    {
      const int64_t KSg = KY * Ds * Dg;
      DevBuf t(Da_ * KSg * sizeof(double), st), td = tbuf(Da_ * KSg);
      run2(ST_SQUEEZE, G(modes({{Da_, 1, KSg}}), modes({{KSg, 1, 1}}), modes({{Da_, Da_, KSg}})), om_d.d(),
           tp(om_dd), Gt.d(), tp(Gtd), t.d(), tp(td));
      run2(ST_SQUEEZE, G(modes({{Dg, 1, Dg}}), modes({{Dg, 1, 1}}), modes({{Da_ * KY * Ds, Dg, Dg}})), t.d(),
           tp(td), Gt.d(), tp(Gtd), om_y.d(), tp(om_yd));
    }
    {
      const int64_t KSg = KX * Ds * Dg;
      DevBuf t(Da_ * KSg * sizeof(double), st), td = tbuf(Da_ * KSg);
      run2(ST_SQUEEZE, G(modes({{Da_, 1, KSg}}), modes({{KSg, 1, 1}}), modes({{Da_, Da_, KSg}})), om_a.d(),
           tp(om_ad), F.d(), tp(Fd), t.d(), tp(td));
      run2(ST_SQUEEZE, G(modes({{Dg, 1, Dg}}), modes({{Dg, 1, 1}}), modes({{Da_ * KX * Ds, Dg, Dg}})), t.d(),
           tp(td), F.d(), tp(Fd), om_x.d(), tp(om_xd));
    }
    // Fy[a,kX,s,g'] = sum_g F[..,g] Om_Y[g,g'];  Gx likewise with Om_X
    DevBuf Fy(Da_ * KX * Ds * Dg * sizeof(double), st), Gx(Da_ * KY * Ds * Dg * sizeof(double), st);
    DevBuf Fyd = tbuf(Da_ * KX * Ds * Dg), Gxd = tbuf(Da_ * KY * Ds * Dg);
    run2(ST_SQUEEZE, G(modes({{Da_ * KX * Ds, Dg, Dg}}), modes({{Dg, 1, 1}}), modes({{Dg, 1, Dg}})), F.d(),
         tp(Fd), om_y.d(), tp(om_yd), Fy.d(), tp(Fyd));
    run2(ST_SQUEEZE, G(modes({{Da_ * KY * Ds, Dg, Dg}}), modes({{Dg, 1, 1}}), modes({{Dg, 1, Dg}})), Gt.d(),
         tp(Gtd), om_x.d(), tp(om_xd), Gx.d(), tp(Gxd));

    const int64_t P = Ds * Ds;
    std::vector<DevBuf> rhoL(d - 1), rhoR(d - 1), rhoLd(d - 1), rhoRd(d - 1);
    // separate leg (position d-1)
    {
      DevBuf eps(Ds * Da_ * Ds * Da_ * sizeof(double), st), phi(Da_ * Ds * Da_ * Ds * sizeof(double), st);
      DevBuf epsd = tbuf(Ds * Da_ * Ds * Da_), phid = tbuf(Da_ * Ds * Da_ * Ds);
      run2(ST_SQUEEZE,
           G(modes({{Ds * Da_, 1, Ds * Da_}}), modes({{Ds * Da_, 1, 1}}), modes({{D0 * KA, Ds * Da_, Ds * Da_}})),
           E.d(), tp(Ed), E.d(), tp(Ed), eps.d(), tp(epsd));
      run2(ST_SQUEEZE,
           G(modes({{Da_, KX * Ds * Dg, Ds * Da_ * Ds}, {Ds, Dg, Da_ * Ds}}),
             modes({{Da_, KX * Ds * Dg, Ds}, {Ds, Dg, 1}}), modes({{KX, Ds * Dg, Ds * Dg}, {Dg, 1, 1}})),
           Fy.d(), tp(Fyd), F.d(), tp(Fd), phi.d(), tp(phid));
      rhoL[d - 2] = DevBuf(P * P * sizeof(double), st);
      rhoLd[d - 2] = tbuf(P * P);
      run2(ST_SQUEEZE,
           G(modes({{Ds, Da_ * Ds * Da_, Ds * Ds * Ds}, {Ds, Da_, Ds}}),
             modes({{Ds, Da_ * Ds, Ds * Ds}, {Ds, 1, 1}}),
             modes({{Da_, Ds * Da_, Ds * Da_ * Ds}, {Da_, 1, Ds}})),
           eps.d(), tp(epsd), phi.d(), tp(phid), rhoL[d - 2].d(), tp(rhoLd[d - 2]));
      DevBuf gam(Da_ * Ds * Da_ * Ds * sizeof(double), st), eta(Ds * Da_ * Ds * Da_ * sizeof(double), st);
      DevBuf gamd = tbuf(Da_ * Ds * Da_ * Ds), etad = tbuf(Ds * Da_ * Ds * Da_);
      run2(ST_SQUEEZE,
           G(modes({{Da_, KY * Ds * Dg, Ds * Da_ * Ds}, {Ds, Dg, Da_ * Ds}}),
             modes({{Da_, KY * Ds * Dg, Ds}, {Ds, Dg, 1}}), modes({{KY, Ds * Dg, Ds * Dg}, {Dg, 1, 1}})),
           Gx.d(), tp(Gxd), Gt.d(), tp(Gtd), gam.d(), tp(gamd));
      run2(ST_SQUEEZE,
           G(modes({{Ds * Da_, 1, Ds * Da_}}), modes({{Ds * Da_, 1, 1}}), modes({{D0 * KD, Ds * Da_, Ds * Da_}})),
           H.d(), tp(Hd), H.d(), tp(Hd), eta.d(), tp(etad));
      rhoR[d - 2] = DevBuf(P * P * sizeof(double), st);
      rhoRd[d - 2] = tbuf(P * P);
      // rho_R[(a,b),(a',b')] = sum_{b,b'} gam[be,a,be',a'] eta[b,be,b',be']
      run2(ST_SQUEEZE,
           G(modes({{Ds, Da_ * Ds, Ds * Ds * Ds}, {Ds, 1, Ds}}),
             modes({{Ds, Da_ * Ds * Da_, Ds * Ds}, {Ds, Da_, 1}}),
             modes({{Da_, Ds * Da_ * Ds, Ds * Da_}, {Da_, Ds, 1}})),
           gam.d(), tp(gamd), eta.d(), tp(etad), rhoR[d - 2].d(), tp(rhoRd[d - 2]));
    }
    if (g > 0 && p.method == TATRG_ATRG) {
      // ATRG: the group isometries I..L are identities, so the pair Gram of group leg nu is
      // the environment traced over the other group leg z.  With
      //   Q_E[x,a,y,b] = sum_{i0,z,s} E[i0,(x,z),s,a] E[i0,(y,z),s,b],
      //   Q_F[a,x,b,y] = sum_{z,s,g} Fy[a,(x,z),s,g] F[b,(y,z),s,g],
      // rho_L[(x,x'),(y,y')] = sum_{a,b} Q_E[x,a,y,b] Q_F[a,x',b,y'], and rho_R likewise from
      // Gx, G and H: chi^4 intermediates and O(chi^7) work in place of the chi^8 environment
      // that the general triad contraction below would build for k = chi^2 (the same sums).
      for (int nu = 1; nu <= g; ++nu) {
        const int64_t Dn = D[nu], Dz = Gd / Dn;
        const int64_t snu = prod(D, nu + 1, 1 + g);  // stride of leg nu in the group index
        const int64_t sz = nu == 1 ? 1 : Dn;          // stride of the other group leg (g == 2)
        const int64_t Pn = Dn * Dn, QQ = Dn * Da_ * Dn * Da_;
        DevBuf qe(QQ * sizeof(double), st), qf(QQ * sizeof(double), st);
        DevBuf qed = tbuf(QQ), qfd = tbuf(QQ);
        run2(ST_SQUEEZE,
             G(modes({{Dn, snu * Ds * Da_, Da_ * Dn * Da_}, {Da_, 1, Dn * Da_}}),
               modes({{Dn, snu * Ds * Da_, Da_}, {Da_, 1, 1}}),
               modes({{D0, KA * Ds * Da_, KA * Ds * Da_}, {Dz, sz * Ds * Da_, sz * Ds * Da_}, {Ds, Da_, Da_}})),
             E.d(), tp(Ed), E.d(), tp(Ed), qe.d(), tp(qed));
        run2(ST_SQUEEZE,
             G(modes({{Da_, KX * Ds * Dg, Dn * Da_ * Dn}, {Dn, snu * Ds * Dg, Da_ * Dn}}),
               modes({{Da_, KX * Ds * Dg, Dn}, {Dn, snu * Ds * Dg, 1}}),
               modes({{Dz, sz * Ds * Dg, sz * Ds * Dg}, {Ds * Dg, 1, 1}})),
             Fy.d(), tp(Fyd), F.d(), tp(Fd), qf.d(), tp(qfd));
        // rho[x,x',y,y'] = sum_{a,b} Q1[x,a,y,b] Q2[a,x',b,y'] (row-major (x,x') x (y,y'))
        const GemmDesc pair = G(modes({{Dn, Da_ * Dn * Da_, Dn * Dn * Dn}, {Dn, Da_, Dn}}),
                                modes({{Dn, Da_ * Dn, Dn * Dn}, {Dn, 1, 1}}),
                                modes({{Da_, Dn * Da_, Dn * Da_ * Dn}, {Da_, 1, Dn}}));
        rhoL[nu - 1] = DevBuf(Pn * Pn * sizeof(double), st);
        rhoLd[nu - 1] = tbuf(Pn * Pn);
        run2(ST_SQUEEZE, pair, qe.d(), tp(qed), qf.d(), tp(qfd), rhoL[nu - 1].d(), tp(rhoLd[nu - 1]));
        // Q_G[x,b,y,c] = sum_{z,s,g} Gx[b,(x,z),s,g] G[c,(y,z),s,g]
        run2(ST_SQUEEZE,
             G(modes({{Dn, snu * Ds * Dg, Da_ * Dn * Da_}, {Da_, KY * Ds * Dg, Dn * Da_}}),
               modes({{Dn, snu * Ds * Dg, Da_}, {Da_, KY * Ds * Dg, 1}}),
               modes({{Dz, sz * Ds * Dg, sz * Ds * Dg}, {Ds * Dg, 1, 1}})),
             Gx.d(), tp(Gxd), Gt.d(), tp(Gtd), qe.d(), tp(qed));
        // Q_H[b,x,c,y] = sum_{j0,z,s} H[j0,(x,z),s,b] H[j0,(y,z),s,c]
        run2(ST_SQUEEZE,
             G(modes({{Da_, 1, Dn * Da_ * Dn}, {Dn, snu * Ds * Da_, Da_ * Dn}}),
               modes({{Da_, 1, Dn}, {Dn, snu * Ds * Da_, 1}}),
               modes({{D0, KD * Ds * Da_, KD * Ds * Da_}, {Dz, sz * Ds * Da_, sz * Ds * Da_}, {Ds, Da_, Da_}})),
             H.d(), tp(Hd), H.d(), tp(Hd), qf.d(), tp(qfd));
        rhoR[nu - 1] = DevBuf(Pn * Pn * sizeof(double), st);
        rhoRd[nu - 1] = tbuf(Pn * Pn);
        run2(ST_SQUEEZE, pair, qe.d(), tp(qed), qf.d(), tp(qfd), rhoR[nu - 1].d(), tp(rhoRd[nu - 1]));
      }
    } else if (g > 0) {
      // Env_L[kA,kA',kX,kX'] = sum_{a,a'} P_E[kA,kA',a,a'] P_F[a,a',kX,kX']
      DevBuf pe(KA * KA * Da_ * Da_ * sizeof(double), st), pf(Da_ * Da_ * KX * KX * sizeof(double), st);
      DevBuf ped = tbuf(KA * KA * Da_ * Da_), pfd = tbuf(Da_ * Da_ * KX * KX);
      run2(ST_SQUEEZE,
           G(modes({{KA, Ds * Da_, KA * Da_ * Da_}, {Da_, 1, Da_}}), modes({{KA, Ds * Da_, Da_ * Da_}, {Da_, 1, 1}}),
             modes({{D0, KA * Ds * Da_, KA * Ds * Da_}, {Ds, Da_, Da_}})),
           E.d(), tp(Ed), E.d(), tp(Ed), pe.d(), tp(ped));
      run2(ST_SQUEEZE,
           G(modes({{Da_, KX * Ds * Dg, Da_ * KX * KX}, {KX, Ds * Dg, KX}}),
             modes({{Da_, KX * Ds * Dg, KX * KX}, {KX, Ds * Dg, 1}}), modes({{Ds * Dg, 1, 1}})),
           Fy.d(), tp(Fyd), F.d(), tp(Fd), pf.d(), tp(pfd));
      DevBuf envL(KA * KA * KX * KX * sizeof(double), st), envLd = tbuf(KA * KA * KX * KX);
      run2(ST_SQUEEZE,
           G(modes({{KA * KA, Da_ * Da_, KX * KX}}), modes({{KX * KX, 1, 1}}), modes({{Da_ * Da_, 1, KX * KX}})),
           pe.d(), tp(ped), pf.d(), tp(pfd), envL.d(), tp(envLd));
      DevBuf pg(KY * KY * Da_ * Da_ * sizeof(double), st), ph(Da_ * Da_ * KD * KD * sizeof(double), st);
      DevBuf pgd = tbuf(KY * KY * Da_ * Da_), phd = tbuf(Da_ * Da_ * KD * KD);
      run2(ST_SQUEEZE,
           G(modes({{KY, Ds * Dg, KY * Da_ * Da_}, {Da_, KY * Ds * Dg, Da_}}),
             modes({{KY, Ds * Dg, Da_ * Da_}, {Da_, KY * Ds * Dg, 1}}), modes({{Ds * Dg, 1, 1}})),
           Gx.d(), tp(Gxd), Gt.d(), tp(Gtd), pg.d(), tp(pgd));
      run2(ST_SQUEEZE,
           G(modes({{Da_, 1, Da_ * KD * KD}, {KD, Ds * Da_, KD}}), modes({{Da_, 1, KD * KD}, {KD, Ds * Da_, 1}}),
             modes({{D0, KD * Ds * Da_, KD * Ds * Da_}, {Ds, Da_, Da_}})),
           H.d(), tp(Hd), H.d(), tp(Hd), ph.d(), tp(phd));
      DevBuf envR(KY * KY * KD * KD * sizeof(double), st), envRd = tbuf(KY * KY * KD * KD);
      run2(ST_SQUEEZE,
           G(modes({{KY * KY, Da_ * Da_, KD * KD}}), modes({{KD * KD, 1, 1}}), modes({{Da_ * Da_, 1, KD * KD}})),
           pg.d(), tp(pgd), ph.d(), tp(phd), envR.d(), tp(envRd));
      for (int nu = 1; nu <= g; ++nu) {
        const int64_t Dn = D[nu];
        const int64_t Dz = Gd / Dn;  // product of the other group legs (1 when g == 1)
        // stride of leg nu and of the others inside the group index (row-major group legs)
        const int64_t snu = prod(D, nu + 1, 1 + g);
        auto pairgram = [&](const DMat& U, const DMat& Ud_, int64_t K, DevBuf& out, DevBuf& outd) {
          out = DevBuf(Dn * Dn * K * K * sizeof(double), st);
          outd = tbuf(Dn * Dn * K * K);
          // out[a,a',k,k'] = sum_z U[(..a..z..),k] U[(..a'..z..),k']
          ModeIdx kz;
          if (g == 1) kz = modes({});
          else if (nu == 1) kz = modes({{Dz, K, K}});        // z = leg 2, stride K
          else kz = modes({{Dz, Dn * K, Dn * K}});           // z = leg 1, stride D2*K
          run2(ST_SQUEEZE,
               G(modes({{Dn, snu * K, Dn * K * K}, {K, 1, K}}), modes({{Dn, snu * K, K * K}, {K, 1, 1}}), kz),
               U.p(), tpm(Ud_), U.p(), tpm(Ud_), out.d(), tp(outd));
        };
        DevBuf ii, jj, kk, ll, iid, jjd, kkd, lld;
        pairgram(UA, UAd, KA, ii, iid);
        pairgram(UX, UXd, KX, jj, jjd);
        pairgram(UY, UYd, KY, kk, kkd);
        pairgram(UD, UDd, KD, ll, lld);
        const int64_t Pn = Dn * Dn;
        DevBuf t(Pn * KX * KX * sizeof(double), st), td = tbuf(Pn * KX * KX);
        run2(ST_SQUEEZE,
             G(modes({{Pn, KA * KA, KX * KX}}), modes({{KX * KX, 1, 1}}), modes({{KA * KA, 1, KX * KX}})),
             ii.d(), tp(iid), envL.d(), tp(envLd), t.d(), tp(td));
        rhoL[nu - 1] = DevBuf(Pn * Pn * sizeof(double), st);
        rhoLd[nu - 1] = tbuf(Pn * Pn);
        run2(ST_SQUEEZE,
             G(modes({{Dn, Dn * KX * KX, Dn * Dn * Dn}, {Dn, KX * KX, Dn}}),
               modes({{Dn, Dn * KX * KX, Dn * Dn}, {Dn, KX * KX, 1}}), modes({{KX * KX, 1, 1}})),
             t.d(), tp(td), jj.d(), tp(jjd), rhoL[nu - 1].d(), tp(rhoLd[nu - 1]));
        DevBuf t2(Pn * KD * KD * sizeof(double), st), t2d = tbuf(Pn * KD * KD);
        run2(ST_SQUEEZE,
             G(modes({{Pn, KY * KY, KD * KD}}), modes({{KD * KD, 1, 1}}), modes({{KY * KY, 1, KD * KD}})),
             kk.d(), tp(kkd), envR.d(), tp(envRd), t2.d(), tp(t2d));
        rhoR[nu - 1] = DevBuf(Pn * Pn * sizeof(double), st);
        rhoRd[nu - 1] = tbuf(Pn * Pn);
        run2(ST_SQUEEZE,
             G(modes({{Dn, Dn * KD * KD, Dn * Dn * Dn}, {Dn, KD * KD, Dn}}),
               modes({{Dn, Dn * KD * KD, Dn * Dn}, {Dn, KD * KD, 1}}), modes({{KD * KD, 1, 1}})),
             t2.d(), tp(t2d), ll.d(), tp(lld), rhoR[nu - 1].d(), tp(rhoRd[nu - 1]));
      }
    }
    // square-root factors of the 2(d - 1) Grams; without tangents they are independent and
    // run concurrently
    std::vector<DMat> RtLs(d - 1), RtRs(d - 1), RtLds(d - 1), RtRds(d - 1);
    if (!T) {
      std::vector<Task> tasks;
      for (int nu = 1; nu <= d - 1; ++nu) {
        const int64_t Pn = D[nu] * D[nu];
        tasks.push_back([&, nu, Pn](Engine& E) {
          factor(E, rhoL[nu - 1].d(), Pn, KIND_SQ_LEFT + nu - 1, RtLs[nu - 1]);
          RtLs[nu - 1].buf.rebind(st);
        });
        tasks.push_back([&, nu, Pn](Engine& E) {
          factor(E, rhoR[nu - 1].d(), Pn, KIND_SQ_RIGHT + nu - 1, RtRs[nu - 1]);
          RtRs[nu - 1].buf.rebind(st);
        });
      }
      concurrent(tasks);
    } else {
      for (int nu = 1; nu <= d - 1; ++nu) {
        const int64_t Pn = D[nu] * D[nu];
        factor(eng, rhoL[nu - 1].d(), Pn, KIND_SQ_LEFT + nu - 1, RtLs[nu - 1], tp(rhoLd[nu - 1]), &RtLds[nu - 1]);
        factor(eng, rhoR[nu - 1].d(), Pn, KIND_SQ_RIGHT + nu - 1, RtRs[nu - 1], tp(rhoRd[nu - 1]), &RtRds[nu - 1]);
      }
    }
    // oblique projectors: C = R_L R_R^T = U S V^T, M = R_R^T V_k S^-1/2, N = S^-1/2 U_k^T R_L
    for (int nu = 1; nu <= d - 1; ++nu) {
      const int64_t Dn = D[nu], Pn = Dn * Dn;
      DMat& RtL = RtLs[nu - 1];
      DMat& RtR = RtRs[nu - 1];
      DMat& RtLd = RtLds[nu - 1];
      DMat& RtRd = RtRds[nu - 1];
      const int64_t kL = RtL.cols, kR = RtR.cols;
      DevBuf C(kL * kR * sizeof(double), st);
      eng.mm(kL, kR, Pn, RtL.p(), kL, true, RtR.p(), kR, false, C.d(), kR);
      SvdResult cs = eng.svd(C.d(), kL, kR);
      const int64_t k = multiplet_cut(cs.s, keep_count(cs.s, 1e-12, chi()), tau);
      TATRG_CHECK(k >= 1, TATRG_ENUMERIC, "squeezer core is zero");
      spec_sq[nu - 1] = cs.s;
      std::vector<double> v(cs.s.begin(), cs.s.begin() + k);
      for (auto& x : v) x = 1.0 / std::sqrt(x);
      DevBuf isq = eng.upload(v);
      Ms[nu - 1].buf = dalloc(Pn * k, st);
      Ms[nu - 1].rows = Pn;
      Ms[nu - 1].cols = k;
      Nts[nu - 1].buf = dalloc(Pn * k, st);
      Nts[nu - 1].rows = Pn;
      Nts[nu - 1].cols = k;
      eng.mm(Pn, k, kR, RtR.p(), kR, false, cs.V.p(), cs.V.cols, false, Ms[nu - 1].p(), k);
      eng.mm(Pn, k, kL, RtL.p(), kL, false, cs.U.p(), cs.U.cols, false, Nts[nu - 1].p(), k);
      if (T) {
        // dC = dR_L^T R_R + R_L^T dR_R;  d(s^-1/2) = -s^-3/2 ds / 2
        DevBuf Cd(kL * kR * sizeof(double), st);
        eng.mm(kL, kR, Pn, RtLd.p(), kL, true, RtR.p(), kR, false, Cd.d(), kR);
        eng.mm(kL, kR, Pn, RtL.p(), kL, true, RtRd.p(), kR, false, Cd.d(), kR, 1.0, 1.0);
        Engine::SvdTan ct = eng.svd_tan(Cd.d(), kL, kR, cs, int(k), multiplet_groups(cs.s, tau));
        std::vector<double> dv(k);
        for (int64_t i = 0; i < k; ++i) dv[i] = -0.5 * ct.s[i] * v[i] * v[i] * v[i];
        DevBuf isqd = eng.upload(dv);
        for (int side = 0; side < 2; ++side) {
          DMat& out = side == 0 ? Ms[nu - 1] : Nts[nu - 1];
          DMat& outd = side == 0 ? Msd[nu - 1] : Ntsd[nu - 1];
          const DMat& R = side == 0 ? RtR : RtL;
          const DMat& Rd = side == 0 ? RtRd : RtLd;
          const DMat& W = side == 0 ? cs.V : cs.U;
          const DMat& Wd = side == 0 ? ct.V : ct.U;
          const int64_t kk = side == 0 ? kR : kL;
          outd.buf = dalloc(Pn * k, st);
          outd.rows = Pn;
          outd.cols = k;
          eng.mm(Pn, k, kk, Rd.p(), kk, false, W.p(), W.cols, false, outd.p(), k);
          eng.mm(Pn, k, kk, R.p(), kk, false, Wd.p(), k, false, outd.p(), k, 1.0, 1.0);
          scale_axis_tan(out.p(), outd.p(), isq.d(), isqd.d(), Pn, k, 1, 1, st);
        }
      } else {
        scale_axis(Ms[nu - 1].p(), isq.d(), Pn, k, 1, 1, st);
        scale_axis(Nts[nu - 1].p(), isq.d(), Pn, k, 1, 1, st);
      }
      canonical_cols(Ms[nu - 1].p(), Pn, int(k), cs.s, Nts[nu - 1].p(), Pn, false, tpm(Msd[nu - 1]),
                     tpm(Ntsd[nu - 1]));
      Kn[nu - 1] = k;
      TATRG_CUDA(cudaStreamSynchronize(st));
    }
  }

  // ============================ contraction (Eqs. 6-7) ============================
  tm.mark(3);
  stage_prec(ST_CONTRACT);
  const int64_t Ks = Kn[d - 2];
  const int64_t Kg = g > 0 ? prod(Kn, 0, g) : 1;
  const int64_t rowsN = D0 * Kg * Ks;  // rows of Phi / Psi: (i0, k_1..k_g, k_sep)
  DMat phi, psi, phid, psid;
  // One side of the contraction; the tangent operands (null outside tangent mode) follow
  // their primal ones.
  auto contract_side = [&](const DevBuf& E_, const DevBuf& Ed_, const DevBuf& F_, const DevBuf& Fd_,
                           int64_t KA_, int64_t KX_, const DMat& I_, const DMat& Id_, const DMat& J_,
                           const DMat& Jd_, const std::vector<DMat>& Ws, const std::vector<DMat>& Wsd,
                           DMat& out, DMat& outd) {
    // C1: em[i0,kA,a,b,k] = sum_a' E[i0,kA,a',a] W_sep[(a',b),k]
    DevBuf em(D0 * KA_ * Da_ * Ds * Ks * sizeof(double), st), emd = tbuf(D0 * KA_ * Da_ * Ds * Ks);
    run2(ST_CONTRACT,
         G(modes({{D0 * KA_, Ds * Da_, Da_ * Ds * Ks}, {Da_, 1, Ds * Ks}}), modes({{Ds * Ks, 1, 1}}),
           modes({{Ds, Da_, Ds * Ks}})),
         E_.d(), tp(Ed_), Ws[d - 2].p(), tpm(Wsd[d - 2]), em.d(), tp(emd));
    // C2: q[i0,kA,k,kX,g] = sum_{a,b} em[i0,kA,a,b,k] F[a,kX,b,g]
    DevBuf qf(D0 * KA_ * Ks * KX_ * Dg * sizeof(double), st), qfd = tbuf(D0 * KA_ * Ks * KX_ * Dg);
    run2(ST_CONTRACT,
         G(modes({{D0 * KA_, Da_ * Ds * Ks, Ks * KX_ * Dg}, {Ks, 1, KX_ * Dg}}),
           modes({{KX_, Ds * Dg, Dg}, {Dg, 1, 1}}), modes({{Da_, Ds * Ks, KX_ * Ds * Dg}, {Ds, Ks, Dg}})),
         em.d(), tp(emd), F_.d(), tp(Fd_), qf.d(), tp(qfd));
    em.release();
    emd.release();
    // C3: P[kA,kX,k_G] = sum I[a_G,kA] J[b_G,kX] prod_nu W_nu[(a_nu,b_nu),k_nu]
    DevBuf pm(KA_ * KX_ * Kg * sizeof(double), st), pmd = tbuf(KA_ * KX_ * Kg);
    if (g == 0) {
      fill(pm.d(), 1, 1.0, st);
    } else if (g == 1) {
      const int64_t D1 = D[1], K1 = Kn[0];
      DevBuf t1(KA_ * D1 * K1 * sizeof(double), st), t1d = tbuf(KA_ * D1 * K1);
      run2(ST_CONTRACT, G(modes({{KA_, 1, D1 * K1}}), modes({{D1 * K1, 1, 1}}), modes({{D1, KA_, D1 * K1}})),
           I_.p(), tpm(Id_), Ws[0].p(), tpm(Wsd[0]), t1.d(), tp(t1d));
      run2(ST_CONTRACT,
           G(modes({{KA_, D1 * K1, KX_ * K1}, {K1, 1, 1}}), modes({{KX_, 1, K1}}), modes({{D1, K1, KX_}})),
           t1.d(), tp(t1d), J_.p(), tpm(Jd_), pm.d(), tp(pmd));
    } else {
      const int64_t D1 = D[1], D2 = D[2], K1 = Kn[0], K2 = Kn[1];
      DevBuf t1(D2 * KA_ * D1 * K1 * sizeof(double), st), t2(KA_ * D1 * K1 * D2 * K2 * sizeof(double), st);
      DevBuf t1d = tbuf(D2 * KA_ * D1 * K1), t2d = tbuf(KA_ * D1 * K1 * D2 * K2);
      run2(ST_CONTRACT,
           G(modes({{D2 * KA_, 1, D1 * K1}}), modes({{D1 * K1, 1, 1}}), modes({{D1, D2 * KA_, D1 * K1}})),
           I_.p(), tpm(Id_), Ws[0].p(), tpm(Wsd[0]), t1.d(), tp(t1d));
      run2(ST_CONTRACT,
           G(modes({{KA_ * D1 * K1, 1, D2 * K2}}), modes({{D2 * K2, 1, 1}}), modes({{D2, KA_ * D1 * K1, D2 * K2}})),
           t1.d(), tp(t1d), Ws[1].p(), tpm(Wsd[1]), t2.d(), tp(t2d));
      run2(ST_CONTRACT,
           G(modes({{KA_, D1 * K1 * D2 * K2, KX_ * K1 * K2}, {K1, D2 * K2, K2}, {K2, 1, 1}}),
             modes({{KX_, 1, K1 * K2}}), modes({{D1, K1 * D2 * K2, D2 * KX_}, {D2, K2, KX_}})),
           t2.d(), tp(t2d), J_.p(), tpm(Jd_), pm.d(), tp(pmd));
    }
    // C4: out[i0,k_G,k,g] = sum_{kA,kX} q[i0,kA,k,kX,g] P[kA,kX,k_G]
    out.buf = dalloc(rowsN * Dg, st);
    out.rows = rowsN;
    out.cols = Dg;
    if (T) {
      outd.buf = dalloc(rowsN * Dg, st);
      outd.rows = rowsN;
      outd.cols = Dg;
    }
    run2(ST_CONTRACT,
         G(modes({{D0, KA_ * Ks * KX_ * Dg, Kg * Ks * Dg}, {Ks, KX_ * Dg, Dg}, {Dg, 1, 1}}),
           modes({{Kg, 1, Ks * Dg}}), modes({{KA_, Ks * KX_ * Dg, KX_ * Kg}, {KX_, Dg, Kg}})),
         qf.d(), tp(qfd), pm.d(), g == 0 ? nullptr : tp(pmd), out.p(), tpm(outd));
  };
  contract_side(E, Ed, F, Fd, KA, KX, UA, UAd, UX, UXd, Ms, Msd, phi, phid);
  // Psi: the same chain with H (for E), G (for F), L, K and the transposed N's; H carries
  // the backward leg j0(n) and L the group legs of site n, so (kD, kY) take the roles of
  // (kA, kX) with the pair order (a, b) = (leg at n+1^, leg at n) kept by N^T.
  {
    // hn[j0,kD,be,a,k] = sum_b H[j0,kD,b,be] N_sep[k,(a,b)]
    DevBuf hn(D0 * KD * Da_ * Ds * Ks * sizeof(double), st), hnd = tbuf(D0 * KD * Da_ * Ds * Ks);
    run2(ST_CONTRACT,
         G(modes({{D0 * KD, Ds * Da_, Da_ * Ds * Ks}, {Da_, 1, Ds * Ks}}), modes({{Ds, Ds * Ks, Ks}, {Ks, 1, 1}}),
           modes({{Ds, Da_, Ks}})),
         H.d(), tp(Hd), Nts[d - 2].p(), tpm(Ntsd[d - 2]), hn.d(), tp(hnd));
    DevBuf qp(D0 * KD * Ks * KY * Dg * sizeof(double), st), qpd = tbuf(D0 * KD * Ks * KY * Dg);
    run2(ST_CONTRACT,
         G(modes({{D0 * KD, Da_ * Ds * Ks, Ks * KY * Dg}, {Ks, 1, KY * Dg}}),
           modes({{KY, Ds * Dg, Dg}, {Dg, 1, 1}}), modes({{Da_, Ds * Ks, KY * Ds * Dg}, {Ds, Ks, Dg}})),
         hn.d(), tp(hnd), Gt.d(), tp(Gtd), qp.d(), tp(qpd));
    hn.release();
    hnd.release();
    // P'[kY,kD,k_G] = sum K[a_G,kY] L[b_G,kD] prod N_nu[k,(a,b)]
    DevBuf pm(KY * KD * Kg * sizeof(double), st), pmd = tbuf(KY * KD * Kg);
    if (g == 0) {
      fill(pm.d(), 1, 1.0, st);
    } else if (g == 1) {
      const int64_t D1 = D[1], K1 = Kn[0];
      DevBuf t1(KY * D1 * K1 * sizeof(double), st), t1d = tbuf(KY * D1 * K1);
      run2(ST_CONTRACT, G(modes({{KY, 1, D1 * K1}}), modes({{D1 * K1, 1, 1}}), modes({{D1, KY, D1 * K1}})),
           UY.p(), tpm(UYd), Nts[0].p(), tpm(Ntsd[0]), t1.d(), tp(t1d));
      run2(ST_CONTRACT,
           G(modes({{KY, D1 * K1, KD * K1}, {K1, 1, 1}}), modes({{KD, 1, K1}}), modes({{D1, K1, KD}})),
           t1.d(), tp(t1d), UD.p(), tpm(UDd), pm.d(), tp(pmd));
    } else {
      const int64_t D1 = D[1], D2 = D[2], K1 = Kn[0], K2 = Kn[1];
      DevBuf t1(D2 * KY * D1 * K1 * sizeof(double), st), t2(KY * D1 * K1 * D2 * K2 * sizeof(double), st);
      DevBuf t1d = tbuf(D2 * KY * D1 * K1), t2d = tbuf(KY * D1 * K1 * D2 * K2);
      run2(ST_CONTRACT,
           G(modes({{D2 * KY, 1, D1 * K1}}), modes({{D1 * K1, 1, 1}}), modes({{D1, D2 * KY, D1 * K1}})),
           UY.p(), tpm(UYd), Nts[0].p(), tpm(Ntsd[0]), t1.d(), tp(t1d));
      run2(ST_CONTRACT,
           G(modes({{KY * D1 * K1, 1, D2 * K2}}), modes({{D2 * K2, 1, 1}}), modes({{D2, KY * D1 * K1, D2 * K2}})),
           t1.d(), tp(t1d), Nts[1].p(), tpm(Ntsd[1]), t2.d(), tp(t2d));
      run2(ST_CONTRACT,
           G(modes({{KY, D1 * K1 * D2 * K2, KD * K1 * K2}, {K1, D2 * K2, K2}, {K2, 1, 1}}),
             modes({{KD, 1, K1 * K2}}), modes({{D1, K1 * D2 * K2, D2 * KD}, {D2, K2, KD}})),
           t2.d(), tp(t2d), UD.p(), tpm(UDd), pm.d(), tp(pmd));
    }
    // Psi[j0,k_G,k,g] = sum_{kD,kY} qp[j0,kD,k,kY,g] P'[kY,kD,k_G]
    psi.buf = dalloc(rowsN * Dg, st);
    psi.rows = rowsN;
    psi.cols = Dg;
    if (T) {
      psid.buf = dalloc(rowsN * Dg, st);
      psid.rows = rowsN;
      psid.cols = Dg;
    }
    run2(ST_CONTRACT,
         G(modes({{D0, KD * Ks * KY * Dg, Kg * Ks * Dg}, {Ks, KY * Dg, Dg}, {Dg, 1, 1}}),
           modes({{Kg, 1, Ks * Dg}}), modes({{KD, Ks * KY * Dg, Kg}, {KY, Dg, KD * Kg}})),
         qp.d(), tp(qpd), pm.d(), g == 0 ? nullptr : tp(pmd), psi.p(), tpm(psid));
  }
  E.release();
  F.release();
  Gt.release();
  H.release();
  Ed.release();
  Fd.release();
  Gtd.release();
  Hd.release();

  // ============================ re-split and rotation ============================
  tm.mark(4);
  stage_prec(ST_RESPLIT);
  std::vector<int64_t> newD(d);
  newD[0] = D0;
  for (int nu = 1; nu < d; ++nu) newD[nu] = Kn[nu - 1];
  resplit_and_rotate(phi, psi, rowsN, Dg, newD, T ? &phid : nullptr, T ? &psid : nullptr);
  tm.mark(5);
  TATRG_CUDA(cudaStreamSynchronize(st));
  for (int i = 0; i < ST_N; ++i) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, tm.ev[i], tm.ev[i + 1]);
    info.ms[i] = ms;
    info.flops[i] = flops[i];
  }
  info.step = step;
  for (int i = 0; i < 5; ++i) info.dims[i] = 0;
  for (int i = 0; i < d && i < 4; ++i) info.dims[i] = int(D[i]);
  info.dims[4] = int(Da);
  info.lnc = lnc.back();
  // tensor-core figures of the context's own stream: the factorisations on the worker
  // streams share the GPU with one another, so their event times are not kernel times
  info.kernel_launches = int(eng.stats().launches - launches0 + side_launches);
  info.tc_launches = int(eng.stats().tc_launches - tc0);
  info.tc_flops = eng.stats().flops_tc - tcf0;
  info.tc_ms = eng.stats().drain_ms();
  info.partial_lnz = partial_lnz();
}

void tatrg_ctx::resplit_and_rotate(DMat& phi, DMat& psi, int64_t rows, int64_t Dg,
                                   const std::vector<int64_t>& newD, DMat* phid, DMat* psid) {
  cudaStream_t st = stream;
  const bool T = tan_on;
  flops[ST_RESPLIT] += 8.0 * double(rows) * double(Dg) * double(Dg);
  OrthResult qa, qb;
  DMat qad, qbd, rad, rbd;  // tangents of Q_Phi, Q_Psi, R_Phi, R_Psi
  if (T) {
    Engine::OrthT ta = eng.orth_t(phi.p(), phid->p(), rows, Dg, tau);
    Engine::OrthT tb = eng.orth_t(psi.p(), psid->p(), rows, Dg, tau);
    qa = std::move(ta.o);
    qb = std::move(tb.o);
    qad = std::move(ta.Qd);
    qbd = std::move(tb.Qd);
    rad = std::move(ta.Rd);
    rbd = std::move(tb.Rd);
  } else {
    qa = eng.orth(phi.p(), rows, Dg);
    qb = eng.orth(psi.p(), rows, Dg);
  }
  const int64_t ka = qa.k, kb = qb.k;
  DevBuf Cm(ka * kb * sizeof(double), st);
  eng.mm(ka, kb, Dg, qa.R.p(), Dg, false, qb.R.p(), Dg, true, Cm.d(), kb);
  SvdResult cs = eng.svd(Cm.d(), ka, kb);
  const int64_t Dn = keep_count(cs.s, 1e-14, chi());
  TATRG_CHECK(Dn >= 1, TATRG_ENUMERIC, "coarse tensor is zero");
  double c = 0.0;
  for (int64_t i = 0; i < Dn; ++i) c += cs.s[i] * cs.s[i];
  c = std::sqrt(c);
  TATRG_CHECK(c > 0.0 && std::isfinite(c), TATRG_ENUMERIC, "zero or non-finite norm");
  const int64_t D0 = newD[0];
  const int64_t Kr = rows / D0;  // product of the squeezed legs
  // A'[rot] = Q_Phi U_k with rows (i0, rest) written in rotated order (rest, i0)
  DevBuf An(rows * Dn * sizeof(double), st), Bn(rows * Dn * sizeof(double), st);
  flops[ST_RESPLIT] += 4.0 * double(rows) * double(ka) * double(Dn);
  auto ga = [&](int64_t ldu, double beta) {
    return G(modes({{D0, Kr * ka, Dn}, {Kr, ka, D0 * Dn}}), modes({{Dn, 1, 1}}), modes({{ka, 1, ldu}}), 1.0, beta);
  };
  // B'[a, rot] = (Q_Psi V_k)^T
  auto gb = [&](int64_t ldv, double beta) {
    return G(modes({{D0, Kr * kb, 1}, {Kr, kb, D0}}), modes({{Dn, 1, rows}}), modes({{kb, 1, ldv}}), 1.0, beta);
  };
  eng.gemm(ga(cs.U.cols, 0.0), qa.Q.p(), cs.U.p(), An.d());
  eng.gemm(gb(cs.V.cols, 0.0), qb.Q.p(), cs.V.p(), Bn.d());
  DevBuf And, Bnd;
  std::vector<double> dsv;
  double dc = 0.0;
  if (T) {
    // dC = dR_a R_b^T + R_a dR_b^T;  dA' = dQ_a U + Q_a dU;  dB' = (dQ_b V + Q_b dV)^T
    DevBuf Cmd(ka * kb * sizeof(double), st);
    eng.mm(ka, kb, Dg, rad.p(), Dg, false, qb.R.p(), Dg, true, Cmd.d(), kb);
    eng.mm(ka, kb, Dg, qa.R.p(), Dg, false, rbd.p(), Dg, true, Cmd.d(), kb, 1.0, 1.0);
    Engine::SvdTan ct = eng.svd_tan(Cmd.d(), ka, kb, cs, int(Dn), multiplet_groups(cs.s, tau));
    And = dalloc(rows * Dn, st);
    Bnd = dalloc(rows * Dn, st);
    eng.gemm(ga(cs.U.cols, 0.0), qad.p(), cs.U.p(), And.d());
    eng.gemm(ga(Dn, 1.0), qa.Q.p(), ct.U.p(), And.d());
    eng.gemm(gb(cs.V.cols, 0.0), qbd.p(), cs.V.p(), Bnd.d());
    eng.gemm(gb(Dn, 1.0), qb.Q.p(), ct.V.p(), Bnd.d());
    dsv = ct.s;
    for (int64_t i = 0; i < Dn; ++i) dc += cs.s[i] * dsv[i];
    dc /= c;
  }
  canonical_cols(An.d(), rows, int(Dn), cs.s, Bn.d(), rows, true, T ? And.d() : nullptr,
                 T ? Bnd.d() : nullptr);
  A = std::move(An);
  B = std::move(Bn);
  Da = Dn;
  s.assign(cs.s.begin(), cs.s.begin() + Dn);
  if (T) {
    // s' = s / c:  ds' = ds / c - s dc / c^2;  d ln c = dc / c
    Ad = std::move(And);
    Bd = std::move(Bnd);
    sd.assign(Dn, 0.0);
    for (int64_t i = 0; i < Dn; ++i) sd[i] = dsv[i] / c - s[i] * dc / (c * c);
    lnc_d.push_back(dc / c);
  }
  for (auto& x : s) x /= c;
  spec_s = s;
  upload_s();
  D.assign(newD.begin() + 1, newD.end());
  D.push_back(newD[0]);
  lnc.push_back(std::log(c));
}

// =================================== C ABI ===================================
namespace {
std::mutex g_err_mu;
std::string g_err;

void set_global_err(const std::string& m) {
  std::lock_guard<std::mutex> l(g_err_mu);
  g_err = m;
}

template <class F>
tatrg_status guard(tatrg_ctx* ctx, F&& f) {
  try {
    f();
    return TATRG_OK;
  } catch (const Error& e) {
    if (ctx) ctx->err = e.what();
    else set_global_err(e.what());
    return e.code;
  } catch (const std::exception& e) {
    if (ctx) ctx->err = e.what();
    else set_global_err(e.what());
    return TATRG_ECUDA;
  }
}
}  // namespace

extern "C" {

tatrg_status tatrg_create(const tatrg_params* params, void* cuda_stream, tatrg_ctx** out) {
  return guard(nullptr, [&] {
    TATRG_CHECK(params && out, TATRG_EINVAL, "tatrg_create: null argument");
    TATRG_CHECK(params->chi >= 1 && params->r >= 1 && params->q >= 0, TATRG_EINVAL,
                "tatrg_create: need chi >= 1, r >= 1, q >= 0");
    TATRG_CHECK(params->method == TATRG_ATRG || params->method == TATRG_TRIAD, TATRG_EINVAL,
                "tatrg_create: unknown method");
    TATRG_CHECK(params->precision >= TATRG_FP64 && params->precision <= TATRG_OZAKI, TATRG_EINVAL,
                "tatrg_create: unknown precision");
    TATRG_CHECK(params->early_precision >= 0 && params->early_precision <= TATRG_OZAKI, TATRG_EINVAL,
                "tatrg_create: unknown early precision");
    // The step's buffers come from the device's stream-ordered pool; keep freed blocks in
    // the pool across synchronisations instead of returning them to the driver each time.
    int dev = 0;
    cudaMemPool_t pool;
    TATRG_CUDA(cudaGetDevice(&dev));
    TATRG_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
    uint64_t keep = UINT64_MAX;
    TATRG_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
    *out = new tatrg_ctx(*params, static_cast<cudaStream_t>(cuda_stream));
  });
}

tatrg_status tatrg_init_ising(tatrg_ctx* ctx, double beta, double h, int d) {
  if (!ctx) return TATRG_EINVAL;
  return guard(ctx, [&] {
    TATRG_CHECK(d >= 2 && d <= 4, TATRG_EINVAL, "tatrg_init_ising: d must be 2, 3 or 4");
    TATRG_CHECK(beta > 0.0 && std::isfinite(beta) && std::isfinite(h), TATRG_EINVAL,
                "tatrg_init_ising: need finite beta > 0 and finite h");
    ctx->init_ising(beta, h, d);
  });
}

tatrg_status tatrg_rg_step(tatrg_ctx* ctx, int nsteps) {
  if (!ctx) return TATRG_EINVAL;
  return guard(ctx, [&] {
    TATRG_CHECK(nsteps >= 0, TATRG_EINVAL, "tatrg_rg_step: negative step count");
    TATRG_CHECK(ctx->ready, TATRG_ESTATE, "tatrg_rg_step before tatrg_init_ising");
    for (int i = 0; i < nsteps; ++i) {
      ctx->rg_step();
      TATRG_CHECK(tc_error_flag(true) == 0, TATRG_ETIMEOUT, "a tensor-core pipeline wait timed out");
    }
  });
}

tatrg_status tatrg_lnZ(tatrg_ctx* ctx, double* out) {
  if (!ctx || !out) return TATRG_EINVAL;
  return guard(ctx, [&] {
    TATRG_CHECK(ctx->ready, TATRG_ESTATE, "tatrg_lnZ before tatrg_init_ising");
    double tt = ctx->trace();
    TATRG_CHECK(tt > 0.0 && std::isfinite(tt), TATRG_ENUMERIC, "non-positive final trace");
    *out = ctx->partial_lnz() + std::ldexp(std::log(tt), -ctx->step);
  });
}

tatrg_status tatrg_grad(tatrg_ctx* ctx, double* dlnZ_dbeta, double* dlnZ_dh, double* d2lnZ_dbeta2) {
  if (!ctx || (!dlnZ_dbeta && !dlnZ_dh && !d2lnZ_dbeta2)) return TATRG_EINVAL;
  return guard(ctx, [&] {
    TATRG_CHECK(ctx->ready && ctx->ising, TATRG_ESTATE, "tatrg_grad needs a run started by tatrg_init_ising");
    // One FP64 tangent pass per derivative: the same run (parameters, replica, number of
    // steps) with the tangent of every tensor carried beside it.  The passes are
    // independent; each runs on its own host thread and non-blocking stream.
    auto tangent = [&](double beta, int dir, cudaStream_t s) {
      tatrg_params pp = ctx->p;
      pp.precision = TATRG_FP64;
      tatrg_ctx sub(pp, s);
      sub.replica = ctx->replica;
      sub.tan_on = true;
      sub.tan_dir = dir;
      sub.init_ising(beta, ctx->h0, ctx->d);
      for (int k = 0; k < ctx->step; ++k) sub.rg_step();
      const double tt = sub.trace();
      TATRG_CHECK(tt > 0.0 && std::isfinite(tt), TATRG_ENUMERIC, "non-positive final trace");
      double sum = 0.0, comp = 0.0;  // compensated sum of 2^-k d ln c_k
      for (size_t k = 0; k < sub.lnc_d.size(); ++k) {
        const double y = std::ldexp(sub.lnc_d[k], -int(k)) - comp;
        const double t = sum + y;
        comp = (t - sum) - y;
        sum = t;
      }
      return sum + std::ldexp(sub.trace_tan(tt), -sub.step);
    };
    // second derivative: central difference of the exact first derivative; the computed
    // ln Z / V is only piecewise smooth (ordered bases change where singular values of
    // different symmetry sectors cross), so the step stays small
    const double e = 1e-6 * std::max(1.0, ctx->beta0);
    if (d2lnZ_dbeta2)
      TATRG_CHECK(ctx->beta0 - e > 0.0, TATRG_EINVAL, "tatrg_grad: beta too small for the second derivative");
    struct Pass {
      double beta;
      int dir;
      double out = 0.0;
    };
    std::vector<Pass> passes;
    if (dlnZ_dbeta) passes.push_back({ctx->beta0, 0});
    if (dlnZ_dh) passes.push_back({ctx->beta0, 1});
    if (d2lnZ_dbeta2) {
      passes.push_back({ctx->beta0 + e, 0});
      passes.push_back({ctx->beta0 - e, 0});
    }
    int dev = 0;
    TATRG_CUDA(cudaGetDevice(&dev));
    TATRG_CUDA(cudaStreamSynchronize(ctx->stream));
    std::mutex mu;
    tatrg_status first = TATRG_OK;
    std::string first_msg;
    std::vector<std::thread> pool;
    for (auto& ps : passes) {
      pool.emplace_back([&, pp = &ps]() {
        cudaStream_t s = nullptr;
        try {
          TATRG_CUDA(cudaSetDevice(dev));
          TATRG_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
          pp->out = tangent(pp->beta, pp->dir, s);
        } catch (const Error& err) {
          std::lock_guard<std::mutex> l(mu);
          if (first == TATRG_OK) { first = err.code; first_msg = err.what(); }
        } catch (const std::exception& err) {
          std::lock_guard<std::mutex> l(mu);
          if (first == TATRG_OK) { first = TATRG_ECUDA; first_msg = err.what(); }
        }
        if (s) {
          cudaStreamSynchronize(s);
          cudaStreamDestroy(s);
        }
      });
    }
    for (auto& t : pool) t.join();
    if (first != TATRG_OK) throw Error(first, first_msg);
    size_t i = 0;
    if (dlnZ_dbeta) *dlnZ_dbeta = passes[i++].out;
    if (dlnZ_dh) *dlnZ_dh = passes[i++].out;
    if (d2lnZ_dbeta2) {
      *d2lnZ_dbeta2 = (passes[i].out - passes[i + 1].out) / (2.0 * e);
      i += 2;
    }
    TATRG_CHECK(tc_error_flag(true) == 0, TATRG_ETIMEOUT, "a tensor-core pipeline wait timed out");
  });
}

tatrg_status tatrg_sweep(tatrg_ctx* ctx, const double* betas, int nbeta, double h, int d,
                         int nsteps, double* lnZ_out) {
  return tatrg_sweep_observables(ctx, betas, nbeta, h, d, nsteps, lnZ_out, nullptr);
}

tatrg_status tatrg_sweep_observables(tatrg_ctx* ctx, const double* betas, int nbeta, double h, int d,
                                     int nsteps, double* lnZ_out, double* X_out) {
  if (!ctx || !betas || !lnZ_out || nbeta < 0) return TATRG_EINVAL;
  return guard(ctx, [&] {
    TATRG_CHECK(d >= 2 && d <= 4 && nsteps >= 0, TATRG_EINVAL, "tatrg_sweep: bad d or step count");
    // The temperatures are independent runs.  Worker threads take them in turn, each
    // with its own non-blocking stream and context, so the many small kernels and host
    // decisions of one run overlap with the large contractions of the others.  Run i uses
    // sketch replica i, so the results do not depend on the scheduling.
    const int nw = std::max(1, std::min(nbeta, ctx->p.sweep_workers > 0 ? ctx->p.sweep_workers : 8));
    int dev = 0;
    TATRG_CUDA(cudaGetDevice(&dev));
    tc_available();  // one-time initialisation before the workers start
    TATRG_CUDA(cudaStreamSynchronize(ctx->stream));
    std::atomic<int> next(0);
    std::atomic<bool> failed(false);  // read by every worker between temperatures
    std::mutex mu;
    tatrg_status first = TATRG_OK;
    std::string first_msg;
    auto fail = [&](tatrg_status c, const std::string& m) {
      std::lock_guard<std::mutex> l(mu);
      if (first == TATRG_OK) { first = c; first_msg = m; }
      failed.store(true);
    };
    std::vector<std::thread> pool;
    for (int w = 0; w < nw; ++w) {
      pool.emplace_back([&]() {
        cudaStream_t s = nullptr;
        try {
          TATRG_CUDA(cudaSetDevice(dev));
          TATRG_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
          for (int i = next++; i < nbeta && !failed.load(); i = next++) {
            tatrg_ctx sub(ctx->p, s);
            sub.replica = uint32_t(i);
            sub.init_ising(betas[i], h, d);
            for (int k = 0; k < nsteps; ++k) {
              sub.rg_step();
              if (X_out) X_out[int64_t(i) * nsteps + k] = sub.order_parameter(d - 1);
            }
            double tt = sub.trace();
            TATRG_CHECK(tt > 0.0 && std::isfinite(tt), TATRG_ENUMERIC, "non-positive final trace in sweep");
            lnZ_out[i] = sub.partial_lnz() + std::ldexp(std::log(tt), -sub.step);
          }
        } catch (const Error& e) {
          fail(e.code, e.what());
        } catch (const std::exception& e) {
          fail(TATRG_ECUDA, e.what());
        }
        if (s) {
          cudaStreamSynchronize(s);
          cudaStreamDestroy(s);
        }
      });
    }
    for (auto& t : pool) t.join();
    TATRG_CHECK(tc_error_flag(true) == 0, TATRG_ETIMEOUT, "a tensor-core pipeline wait timed out");
    if (first != TATRG_OK) throw Error(first, first_msg);
  });
}

tatrg_status tatrg_order_parameter(tatrg_ctx* ctx, int leg, double* X) {
  if (!ctx || !X) return TATRG_EINVAL;
  return guard(ctx, [&] {
    TATRG_CHECK(ctx->ready, TATRG_ESTATE, "tatrg_order_parameter before init");
    TATRG_CHECK(leg >= 0 && leg < ctx->d, TATRG_EINVAL, "tatrg_order_parameter: leg out of range");
    *X = ctx->order_parameter(leg);
  });
}

tatrg_status tatrg_spectrum(const tatrg_ctx* ctx, int kind, double* out, int* n) {
  if (!ctx || !n) return TATRG_EINVAL;
  const std::vector<double>* v = nullptr;
  if (kind == 0) v = &ctx->spec_s;
  else if (kind == 1) v = &ctx->spec_sigma;
  else if (kind >= 2 && size_t(kind - 2) < ctx->spec_sq.size()) v = &ctx->spec_sq[kind - 2];
  if (!v || (out && *n < 0)) return TATRG_EINVAL;
  int cap = *n;
  *n = int(v->size());
  if (out) std::memcpy(out, v->data(), sizeof(double) * std::min<size_t>(cap, v->size()));
  return TATRG_OK;
}

tatrg_status tatrg_get_state(const tatrg_ctx* ctx, int* d, int* dims, double* A, double* s, double* B) {
  if (!ctx || !d) return TATRG_EINVAL;
  tatrg_ctx* c = const_cast<tatrg_ctx*>(ctx);
  return guard(c, [&] {
    TATRG_CHECK(ctx->ready, TATRG_ESTATE, "tatrg_get_state before init");
    *d = ctx->d;
    if (dims) {
      for (int i = 0; i < ctx->d; ++i) dims[i] = int(ctx->D[i]);
      dims[ctx->d] = int(ctx->Da);
    }
    const int64_t F = prod(ctx->D, 0, ctx->D.size());
    if (A) TATRG_CUDA(cudaMemcpyAsync(A, ctx->A.d(), F * ctx->Da * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (B) TATRG_CUDA(cudaMemcpyAsync(B, ctx->B.d(), F * ctx->Da * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (s) std::memcpy(s, ctx->s.data(), ctx->Da * sizeof(double));
    TATRG_CUDA(cudaStreamSynchronize(ctx->stream));
  });
}

tatrg_status tatrg_set_state(tatrg_ctx* ctx, int d, const int* dims, const double* A, const double* s,
                             const double* B, int step, double partial_lnz) {
  if (!ctx || !dims || !A || !s || !B) return TATRG_EINVAL;
  return guard(ctx, [&] {
    TATRG_CHECK(d >= 2 && d <= 4 && step >= 0, TATRG_EINVAL, "tatrg_set_state: bad d or step");
    for (int i = 0; i <= d; ++i) TATRG_CHECK(dims[i] >= 1, TATRG_EINVAL, "tatrg_set_state: bad dims");
    for (int i = 0; i < dims[d]; ++i)
      TATRG_CHECK(std::isfinite(s[i]), TATRG_ENUMERIC, "tatrg_set_state: non-finite entry in s");
    std::vector<int64_t> D(dims, dims + d);
    const int64_t F = prod(D, 0, D.size()), Da = dims[d];
    // upload and check into new buffers; the context's state changes only when both pass
    DevBuf nA(F * Da * sizeof(double), ctx->stream), nB(F * Da * sizeof(double), ctx->stream);
    TATRG_CUDA(cudaMemcpyAsync(nA.d(), A, F * Da * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    TATRG_CUDA(cudaMemcpyAsync(nB.d(), B, F * Da * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    DevBuf bad(sizeof(int), ctx->stream);
    TATRG_CUDA(cudaMemsetAsync(bad.d(), 0, sizeof(int), ctx->stream));
    check_finite(nA.d(), F * Da, bad.as<int>(), ctx->stream);
    check_finite(nB.d(), F * Da, bad.as<int>(), ctx->stream);
    int hbad = 0;
    TATRG_CUDA(cudaMemcpyAsync(&hbad, bad.d(), sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    TATRG_CUDA(cudaStreamSynchronize(ctx->stream));
    TATRG_CHECK(hbad == 0, TATRG_ENUMERIC, "tatrg_set_state: non-finite entries in A or B");
    ctx->d = d;
    ctx->D = D;
    ctx->Da = Da;
    ctx->A = std::move(nA);
    ctx->B = std::move(nB);
    ctx->s.assign(s, s + ctx->Da);
    ctx->upload_s();
    ctx->step = step;
    // keep ln c_k so that partial_lnz() reproduces the given sum: put it all in k = 0
    ctx->lnc.assign(step + 1, 0.0);
    ctx->lnc[0] = partial_lnz;
    ctx->ready = true;
    ctx->ising = false;
    TATRG_CUDA(cudaStreamSynchronize(ctx->stream));
  });
}

tatrg_status tatrg_last_step_info(const tatrg_ctx* ctx, tatrg_step_info* out) {
  if (!ctx || !out) return TATRG_EINVAL;
  *out = ctx->info;
  return TATRG_OK;
}

const char* tatrg_last_error(const tatrg_ctx* ctx) {
  if (ctx) return ctx->err.c_str();
  std::lock_guard<std::mutex> l(g_err_mu);
  return g_err.c_str();
}

void tatrg_destroy(tatrg_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  delete ctx;
}

tatrg_status tatrg_gaussian(unsigned long long seed, uint32_t sid, uint32_t replica, int64_t rows,
                            int64_t cols, double* out, void* stream) {
  return guard(nullptr, [&] {
    TATRG_CHECK(out && rows >= 0 && cols >= 0, TATRG_EINVAL, "tatrg_gaussian: bad argument");
    gaussian(seed, sid, replica, rows * cols, out, static_cast<cudaStream_t>(stream));
  });
}

namespace {
GemmDesc desc_of(const tatrg_contraction* c) {
  GemmDesc g;
  g.m = modes({{c->m_ext[0], c->m_sA[0], c->m_sC[0]}, {c->m_ext[1], c->m_sA[1], c->m_sC[1]},
               {c->m_ext[2], c->m_sA[2], c->m_sC[2]}, {c->m_ext[3], c->m_sA[3], c->m_sC[3]}});
  g.n = modes({{c->n_ext[0], c->n_sB[0], c->n_sC[0]}, {c->n_ext[1], c->n_sB[1], c->n_sC[1]},
               {c->n_ext[2], c->n_sB[2], c->n_sC[2]}, {c->n_ext[3], c->n_sB[3], c->n_sC[3]}});
  g.k = modes({{c->k_ext[0], c->k_sA[0], c->k_sB[0]}, {c->k_ext[1], c->k_sA[1], c->k_sB[1]},
               {c->k_ext[2], c->k_sA[2], c->k_sB[2]}, {c->k_ext[3], c->k_sA[3], c->k_sB[3]}});
  for (int i = 0; i < 4; ++i) {
    TATRG_CHECK(c->m_ext[i] >= 1 && c->n_ext[i] >= 1 && c->k_ext[i] >= 1, TATRG_EINVAL,
                "tatrg_contract: extents must be >= 1");
    // caller memory is reached from its base pointer only: offsets never go below it
    TATRG_CHECK(c->m_sA[i] >= 0 && c->m_sC[i] >= 0 && c->n_sB[i] >= 0 && c->n_sC[i] >= 0 &&
                    c->k_sA[i] >= 0 && c->k_sB[i] >= 0,
                TATRG_EINVAL, "tatrg_contract: strides must be non-negative");
  }
  g.alpha = c->alpha;
  g.beta = c->beta;
  return g;
}
}  // namespace

tatrg_status tatrg_contract_sketch(const tatrg_contraction* c, int precision, const double* A,
                                   unsigned long long seed, uint32_t sid, uint32_t replica, double* C,
                                   void* stream) {
  return guard(nullptr, [&] {
    TATRG_CHECK(c && A && C, TATRG_EINVAL, "tatrg_contract_sketch: null argument");
    TATRG_CHECK(precision >= 1 && precision <= 3, TATRG_EINVAL,
                "tatrg_contract_sketch: needs a split precision (1, 2 or 3)");
    const GemmDesc g = desc_of(c);
    Engine e(static_cast<cudaStream_t>(stream));
    e.prec = precision;
    const GaussSrc gs{seed, sid, replica};
    TATRG_CHECK(e.gemm_gauss_b(g, A, gs, C), TATRG_EINVAL,
                "tatrg_contract_sketch: contraction too small for the tensor-core path");
    TATRG_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    TATRG_CHECK(tc_error_flag(true) == 0, TATRG_ETIMEOUT, "a tensor-core pipeline wait timed out");
  });
}

tatrg_status tatrg_contract(const tatrg_contraction* c, int precision, const double* A, const double* B,
                            double* C, void* stream) {
  return guard(nullptr, [&] {
    TATRG_CHECK(c && A && B && C, TATRG_EINVAL, "tatrg_contract: null argument");
    TATRG_CHECK(precision >= 0 && precision <= 4, TATRG_EINVAL, "tatrg_contract: bad precision");
    const GemmDesc g = desc_of(c);
    Engine e(static_cast<cudaStream_t>(stream));
    e.prec = precision;
    e.gemm(g, A, B, C);
    if (precision != 0) {
      TATRG_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
      TATRG_CHECK(tc_error_flag(true) == 0, TATRG_ETIMEOUT, "a tensor-core pipeline wait timed out");
    }
  });
}

tatrg_status tatrg_orth(int precision, int64_t m, int64_t n, const double* Y, double* Q, double* R,
                        int* k, void* stream) {
  return guard(nullptr, [&] {
    TATRG_CHECK(Y && Q && R && k && m >= n && n >= 1 && n <= 1024, TATRG_EINVAL, "tatrg_orth: bad argument");
    TATRG_CHECK(precision >= 0 && precision <= 4, TATRG_EINVAL, "tatrg_orth: bad precision");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Engine e(s);
    e.prec = precision;
    OrthResult o = e.orth(Y, m, n);
    TATRG_CUDA(cudaMemcpyAsync(Q, o.Q.p(), m * o.k * sizeof(double), cudaMemcpyDeviceToDevice, s));
    TATRG_CUDA(cudaMemcpyAsync(R, o.R.p(), int64_t(o.k) * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    TATRG_CUDA(cudaStreamSynchronize(s));
    *k = o.k;
  });
}

tatrg_status tatrg_svd(int64_t m, int64_t n, const double* A, double* U, double* S, double* V, void* stream) {
  return guard(nullptr, [&] {
    TATRG_CHECK(A && U && S && V && m >= n && n >= 1 && n <= 1024, TATRG_EINVAL, "tatrg_svd: bad argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Engine e(s);
    SvdResult r = e.svd(A, m, n);
    TATRG_CUDA(cudaMemcpyAsync(U, r.U.p(), m * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    TATRG_CUDA(cudaMemcpyAsync(S, r.S.d(), n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    TATRG_CUDA(cudaMemcpyAsync(V, r.V.p(), n * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    TATRG_CUDA(cudaStreamSynchronize(s));
  });
}

tatrg_status tatrg_svd_noalloc(int64_t m, int64_t n, const double* A, double* U, double* S, double* V,
                               void* stream) {
  return guard(nullptr, [&] {
    TATRG_CHECK(A && U && S && V, TATRG_EINVAL, "tatrg_svd_noalloc: null argument");
    TATRG_CHECK(n >= 1 && n <= 1024 && m >= n, TATRG_EINVAL, "tatrg_svd_noalloc: need m >= n, 1 <= n <= 1024");
    jacobi_svd_noalloc(A, m, int(n), U, S, V, static_cast<cudaStream_t>(stream));
  });
}

tatrg_status tatrg_philox_words(unsigned long long seed, uint32_t sid, uint32_t replica, uint64_t first,
                                int64_t npairs, uint32_t* out, void* stream) {
  return guard(nullptr, [&] {
    TATRG_CHECK(out && npairs >= 0, TATRG_EINVAL, "tatrg_philox_words: bad argument");
    philox_words(seed, sid, replica, first, npairs, out, static_cast<cudaStream_t>(stream));
  });
}

tatrg_status tatrg_set_barrier_limit_ns(long long limit_ns) {
  return guard(nullptr, [&] {
    TATRG_CHECK(limit_ns >= 0, TATRG_EINVAL, "tatrg_set_barrier_limit_ns: negative limit");
    set_barrier_limit_ns(static_cast<unsigned long long>(limit_ns));
  });
}

tatrg_status tatrg_set_cta_pairs(int mode) {
  return guard(nullptr, [&] {
    TATRG_CHECK(mode >= -1 && mode <= 2, TATRG_EINVAL, "tatrg_set_cta_pairs: mode must be -1, 0, 1 or 2");
    set_pair_mode(mode);
  });
}

}  // extern "C"
