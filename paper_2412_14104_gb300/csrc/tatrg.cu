// The Triad-ATRG RG step on the GPU (Sugimoto & Sasaki, arXiv:2412.14104, Sec. 2) and the
// C ABI of include/tatrg.h.  Every contraction below is one multi-mode GEMM whose modes
// are named after the paper's indices; stage order: bond swap (Eq. 1), triad isometries
// and tensors (Eqs. 2-4), squeezers (Eq. 5), contraction (Eqs. 6-7), re-split.
#include <cmath>
#include <cstring>
#include <atomic>
#include <mutex>
#include <thread>
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

  tatrg_ctx(const tatrg_params& pp, cudaStream_t s) : p(pp), stream(s), eng(s) {
    eng.stats().timing = pp.profile != 0;
  }

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
  }

  // Apply the sign convention to the columns of X (F x n, row-major): v = w^T X with the
  // hashed weights; flip the columns (and those of Y, F2 x n, if given) where v < 0.
  void fix_sign_cols(double* X, int64_t F, int n, double* Y, int64_t F2) {
    DevBuf v(std::max(n, 1) * sizeof(double), stream);
    weighted_colsum(X, F, n, v.d(), stream);
    flip_by_sign(X, F, n, nullptr, 0, v.d(), stream);
    if (Y) flip_by_sign(Y, F2, n, nullptr, 0, v.d(), stream);
  }
  // Same, but Y is n x F2 (flip its rows).
  void fix_sign_cols_rows(double* X, int64_t F, int n, double* Y, int64_t F2) {
    DevBuf v(std::max(n, 1) * sizeof(double), stream);
    weighted_colsum(X, F, n, v.d(), stream);
    flip_by_sign(X, F, n, Y, F2, v.d(), stream);
  }

  // Canonical basis of the columns of X (F x n): the sign rule for single columns and, for
  // each degenerate multiplet of vals, the rotation V_M -> V_M O with O the polar factor
  // of V_M^T W (W: hashed weights).  The same rotation is applied to Y: to its rows when
  // y_rows (Y is n x F2), else to its columns (Y is F2 x n).
  void canonical_cols(double* X, int64_t F, int n, const std::vector<double>& vals, double* Y,
                      int64_t F2, bool y_rows);
  void init_ising(double beta, double h, int dd);
  void rg_step();
  void resplit_and_rotate(DMat& phi, DMat& psi, int64_t rows, int64_t Dg,
                          const std::vector<int64_t>& newD);
  double trace();
  DMat isometry(const double* rho, int64_t Gd, int kind, std::vector<double>* lam_out);
  void factor(const double* rho, int64_t P, int kind, DMat& Rt);
};

// ---------------------------------------------------------------------------------
void tatrg_ctx::canonical_cols(double* X, int64_t F, int n, const std::vector<double>& vals,
                               double* Y, int64_t F2, bool y_rows) {
  if (y_rows) fix_sign_cols_rows(X, F, n, Y, F2);
  else fix_sign_cols(X, F, n, Y, F2);
  const int saved = eng.prec;
  eng.prec = 0;
  for (auto& ab : multiplets(vals, n, tau)) {
    const int a = ab.first, m = ab.second - ab.first;
    TATRG_CHECK(m <= 32, TATRG_ENUMERIC, "degenerate multiplet larger than 32");
    DevBuf G(m * m * sizeof(double), stream), O(m * m * sizeof(double), stream);
    multiplet_overlap(X, F, n, a, m, G.d(), stream);
    SvdResult e = eng.svd(G.d(), m, m);
    eng.mm(m, m, m, e.U.p(), m, false, e.V.p(), m, true, O.d(), m);  // O = U V^T
    DevBuf T(F * m * sizeof(double), stream);
    // X[:, a:a+m] <- X[:, a:a+m] O
    eng.gemm(G_(modes({{F, n, m}}), modes({{m, 1, 1}}), modes({{m, 1, m}})), X + a, O.d(), T.d());
    copy_modes(X + a, T.d(), modes({{F, m, n}, {m, 1, 1}}), 1.0, stream);
    if (Y) {
      DevBuf T2(F2 * m * sizeof(double), stream);
      if (y_rows) {  // Y[a:a+m, :] <- O^T Y[a:a+m, :]
        eng.gemm(G_(modes({{m, 1, F2}}), modes({{F2, 1, 1}}), modes({{m, m, F2}})), O.d(), Y + a * F2, T2.d());
        copy_modes(Y + a * F2, T2.d(), modes({{m * F2, 1, 1}}), 1.0, stream);
      } else {       // Y[:, a:a+m] <- Y[:, a:a+m] O
        eng.gemm(G_(modes({{F2, n, m}}), modes({{m, 1, 1}}), modes({{m, 1, m}})), Y + a, O.d(), T2.d());
        copy_modes(Y + a, T2.d(), modes({{F2, m, n}, {m, 1, 1}}), 1.0, stream);
      }
    }
  }
  eng.prec = saved;
}

void tatrg_ctx::init_ising(double beta, double h, int dd) {
  d = dd;
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
  fix_sign_cols_rows(A.d(), n, int(Da), B.d(), n);
  s.assign(e.s.begin(), e.s.begin() + Da);
  for (auto& x : s) x /= c0;
  upload_s();
  lnc.assign(1, std::log(c0));
  step = 0;
  ready = true;
  TATRG_CUDA(cudaStreamSynchronize(stream));
}

double tatrg_ctx::trace() {
  DevBuf out(sizeof(double), stream);
  trace_asb(A.d(), sdev.d(), B.d(), prod(D, 0, D.size()), int(Da), out.d(), stream);
  return eng.to_host(out.d(), 1)[0];
}

// Leading eigenvectors of a PSD Gram (Eqs. 2-3): exact (k >= G) or RSVD with ell = k.
DMat tatrg_ctx::isometry(const double* rho, int64_t Gd, int kind, std::vector<double>* lam_out) {
  DMat U;
  if (p.method == TATRG_ATRG) {
    U.buf = dalloc(Gd * Gd, stream);
    U.rows = U.cols = Gd;
    fill(U.p(), Gd * Gd, 0.0, stream);
    ModeIdx diag = modes({{Gd, 0, Gd + 1}});
    DevBuf one(sizeof(double), stream);
    fill(one.d(), 1, 1.0, stream);
    copy_modes(U.p(), one.d(), diag, 1.0, stream);
    return U;
  }
  const int64_t k = std::min(width(), Gd);
  SvdResult e;
  if (k >= Gd) {
    e = eng.svd(rho, Gd, Gd);
  } else {
    DevBuf om(Gd * k * sizeof(double), stream);
    gaussian(p.seed, stream_id(step, kind), replica, Gd * k, om.d(), stream);
    e = eng.rsvd_psd(rho, Gd, k, p.q, om.d());
  }
  int keep = keep_count(e.s, 1e-14, k);
  TATRG_CHECK(keep >= 1, TATRG_ENUMERIC, "triad Gram is zero");
  U.buf = dalloc(Gd * keep, stream);
  U.rows = Gd;
  U.cols = keep;
  copy_modes(U.p(), e.U.p(), modes({{Gd, e.U.cols, keep}, {keep, 1, 1}}), 1.0, stream);
  fix_sign_cols(U.p(), Gd, keep, nullptr, 0);
  if (lam_out) *lam_out = e.s;
  return U;
}

// rho ~= R^T R from the leading eigenpairs (exact when ell >= P); returns R^T (P x keep).
void tatrg_ctx::factor(const double* rho, int64_t P, int kind, DMat& Rt) {
  const int64_t ell = std::min(width(), P);
  SvdResult e;
  if (ell >= P) {
    e = eng.svd(rho, P, P);
  } else {
    DevBuf om(P * ell * sizeof(double), stream);
    gaussian(p.seed, stream_id(step, kind), replica, P * ell, om.d(), stream);
    e = eng.rsvd_psd(rho, P, ell, p.q, om.d());
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
  scale_axis(Rt.p(), sqd.d(), P, keep, 1, 1, stream);
  TATRG_CUDA(cudaStreamSynchronize(stream));
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
  tau = split ? 1e-6 : 1e-10;
  auto stage_prec = [&](Stage sg) { eng.prec = (split && (mask >> sg) & 1) ? p.precision : 0; };
  stage_prec(ST_SWAP);
  cudaStream_t st = stream;
  StageTimer tm(st);
  const long launches0 = eng.stats().launches, tc0 = eng.stats().tc_launches;
  const double tcf0 = eng.stats().flops_tc;
  eng.stats().drain_ms();
  for (auto& f : flops) f = 0.0;
  auto count = [&](Stage sg, const GemmDesc& g) {
    flops[sg] += 2.0 * double(g.m.total()) * double(g.n.total()) * double(g.k.total());
  };
  auto run = [&](Stage sg, const GemmDesc& g, const double* a, const double* b, double* c) {
    count(sg, g);
    eng.gemm(g, a, b, c);
  };

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
  scale_axis(As.d(), sdev.d(), D0 * I, Da_, 1, 1, st);  // A[k,i,b] s_b
  scale_axis(Bs.d(), sdev.d(), 1, Da_, D0 * I, 1, st);  // s_a B[a,k,j]
  const int64_t rows = Da_ * I;
  const int64_t ell = std::min(width(), rows);
  SvdResult sw;
  info.swap_exact = 0;
  if (ell >= rows) {
    // dense Mid[(a,i),(b,j)] = sum_k Bs[a,k,j] As[k,i,b], one contraction per (a, b)
    info.swap_exact = 1;
    DevBuf mid(rows * rows * sizeof(double), st);
    for (int64_t a = 0; a < Da_; ++a)
      for (int64_t b = 0; b < Da_; ++b) {
        GemmDesc gm = G(modes({{I, Da_, rows}}), modes({{I, 1, 1}}), modes({{D0, I * Da_, I}}));
        run(ST_SWAP, gm, As.d() + b, Bs.d() + a * D0 * I, mid.d() + a * I * rows + b * I);
      }
    sw = eng.svd(mid.d(), rows, rows);
  } else {
    DevBuf om(rows * ell * sizeof(double), st);
    gaussian(p.seed, stream_id(step, KIND_SWAP), replica, rows * ell, om.d(), st);
    // M X: W[a,k,b,p] = sum_j Bs[a,k,j] X[(b,j),p];  Y[(a,i),p] = sum_{k,b} As[k,i,b] W[a,k,b,p]
    auto apply = [&](const double* X, int64_t w, double* Y) {
      DevBuf W(Da_ * D0 * Da_ * w * sizeof(double), st);
      run(ST_SWAP,
          G(modes({{Da_ * D0, I, Da_ * w}}), modes({{Da_, I * w, w}, {w, 1, 1}}), modes({{I, 1, w}})),
          Bs.d(), X, W.d());
      run(ST_SWAP,
          G(modes({{I, Da_, w}}), modes({{Da_, D0 * Da_ * w, I * w}, {w, 1, 1}}),
            modes({{D0, I * Da_, Da_ * w}, {Da_, 1, w}})),
          As.d(), W.d(), Y);
    };
    // M^T X: W[a,k,b,p] = sum_i As[k,i,b] X[(a,i),p];  Z[(b,j),p] = sum_{a,k} Bs[a,k,j] W[a,k,b,p]
    auto rapply = [&](const double* X, int64_t w, double* Z) {
      DevBuf W(Da_ * D0 * Da_ * w * sizeof(double), st);
      run(ST_SWAP,
          G(modes({{D0, I * Da_, Da_ * w}, {Da_, 1, w}}), modes({{Da_, I * w, D0 * Da_ * w}, {w, 1, 1}}),
            modes({{I, Da_, w}})),
          As.d(), X, W.d());
      run(ST_SWAP,
          G(modes({{I, 1, w}}), modes({{Da_, w, I * w}, {w, 1, 1}}), modes({{Da_ * D0, I, Da_ * w}})),
          Bs.d(), W.d(), Z);
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
    if (nL > ell) {
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
      apply_R(om.d(), ell, W0.p());
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
      if (om.empty()) {
        om = DevBuf(rows * ell * sizeof(double), st);
        gaussian(p.seed, stream_id(step, KIND_SWAP), replica, rows * ell, om.d(), st);
      }
      sw = eng.rsvd(apply, rapply, rows, rows, ell, p.q, om.d());
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
  fix_sign_cols(X.d(), rows, int(Dg), Y.d(), rows);
  std::vector<double> sig(sw.s.begin(), sw.s.begin() + Dg);
  DevBuf sigd(Dg * sizeof(double), st);
  TATRG_CUDA(cudaMemcpyAsync(sigd.d(), sig.data(), Dg * sizeof(double), cudaMemcpyHostToDevice, st));
  As.release();
  Bs.release();

  // ======================== triad isometries and tensors (Eqs. 2-4) ========================
  tm.mark(1);
  stage_prec(ST_TRIAD);
  const int64_t nx = Da_ * Gd * Ds * Dg;  // elements of X (= Y)
  DevBuf Xs(nx * sizeof(double), st), Ys(nx * sizeof(double), st);
  TATRG_CUDA(cudaMemcpyAsync(Xs.d(), X.d(), nx * sizeof(double), cudaMemcpyDeviceToDevice, st));
  TATRG_CUDA(cudaMemcpyAsync(Ys.d(), Y.d(), nx * sizeof(double), cudaMemcpyDeviceToDevice, st));
  scale_axis(Xs.d(), sigd.d(), Da_ * Gd * Ds, Dg, 1, 2, st);
  scale_axis(Ys.d(), sigd.d(), Da_ * Gd * Ds, Dg, 1, 2, st);
  const int64_t GSg = Gd * Ds * Dg;
  DevBuf xi_x(Da_ * Da_ * sizeof(double), st), xi_y(Da_ * Da_ * sizeof(double), st);
  run(ST_TRIAD, G(modes({{Da_, GSg, Da_}}), modes({{Da_, GSg, 1}}), modes({{GSg, 1, 1}})), Xs.d(), X.d(), xi_x.d());
  run(ST_TRIAD, G(modes({{Da_, GSg, Da_}}), modes({{Da_, GSg, 1}}), modes({{GSg, 1, 1}})), Ys.d(), Y.d(), xi_y.d());
  DevBuf rho_a(Gd * Gd * sizeof(double), st), rho_x(Gd * Gd * sizeof(double), st),
      rho_y(Gd * Gd * sizeof(double), st), rho_d(Gd * Gd * sizeof(double), st);
  {
    // t_a[i0,G,s,a'] = sum_a A[i0,G,s,a] Xi_X[a,a'];  rho_A[G,G'] = sum t_a[i0,G,s,a] A[i0,G',s,a]
    DevBuf ta(D0 * Gd * Ds * Da_ * sizeof(double), st);
    run(ST_TRIAD, G(modes({{D0 * Gd * Ds, Da_, Da_}}), modes({{Da_, 1, 1}}), modes({{Da_, 1, Da_}})),
        A.d(), xi_x.d(), ta.d());
    run(ST_TRIAD,
        G(modes({{Gd, Ds * Da_, Gd}}), modes({{Gd, Ds * Da_, 1}}),
          modes({{D0, Gd * Ds * Da_, Gd * Ds * Da_}, {Ds * Da_, 1, 1}})),
        ta.d(), A.d(), rho_a.d());
    // rho_X[G,G'] = sum_{a,s,g} Xs[a,G,s,g] X[a,G',s,g]  (and rho_Y)
    GemmDesc gx = G(modes({{Gd, Ds * Dg, Gd}}), modes({{Gd, Ds * Dg, 1}}),
                    modes({{Da_, GSg, GSg}, {Ds * Dg, 1, 1}}));
    run(ST_TRIAD, gx, Xs.d(), X.d(), rho_x.d());
    run(ST_TRIAD, gx, Ys.d(), Y.d(), rho_y.d());
    // t_d[b',j0,G,s] = sum_b Xi_Y[b,b'] D[b,j0,G,s];  rho_D = sum t_d[b,j0,G,s] D[b,j0,G',s]
    DevBuf td(Da_ * D0 * Gd * Ds * sizeof(double), st);
    const int64_t JGS = D0 * Gd * Ds;
    run(ST_TRIAD, G(modes({{Da_, 1, JGS}}), modes({{JGS, 1, 1}}), modes({{Da_, Da_, JGS}})),
        xi_y.d(), B.d(), td.d());
    run(ST_TRIAD,
        G(modes({{Gd, Ds, Gd}}), modes({{Gd, Ds, 1}}), modes({{Da_ * D0, Gd * Ds, Gd * Ds}, {Ds, 1, 1}})),
        td.d(), B.d(), rho_d.d());
  }
  Xs.release();
  Ys.release();
  DMat UA = isometry(rho_a.d(), Gd, KIND_TRIAD_A, nullptr);
  DMat UX = isometry(rho_x.d(), Gd, KIND_TRIAD_X, nullptr);
  DMat UY = isometry(rho_y.d(), Gd, KIND_TRIAD_Y, nullptr);
  DMat UD = isometry(rho_d.d(), Gd, KIND_TRIAD_D, nullptr);
  const int64_t KA = UA.cols, KX = UX.cols, KY = UY.cols, KD = UD.cols;
  // E[i0,kA,s,a] = sum_G A[i0,G,s,a] UA[G,kA]
  DevBuf E(D0 * KA * Ds * Da_ * sizeof(double), st), F(Da_ * KX * Ds * Dg * sizeof(double), st),
      Gt(Da_ * KY * Ds * Dg * sizeof(double), st), H(D0 * KD * Ds * Da_ * sizeof(double), st);
  run(ST_TRIAD,
      G(modes({{D0, Gd * Ds * Da_, KA * Ds * Da_}, {Ds * Da_, 1, 1}}), modes({{KA, 1, Ds * Da_}}),
        modes({{Gd, Ds * Da_, KA}})),
      A.d(), UA.p(), E.d());
  // F[a,kX,s,g] = sum_G X[a,G,s,g] UX[G,kX] sigma_g ;  G[b,kY,s,g] likewise with Y
  run(ST_TRIAD,
      G(modes({{Da_, GSg, KX * Ds * Dg}, {Ds * Dg, 1, 1}}), modes({{KX, 1, Ds * Dg}}),
        modes({{Gd, Ds * Dg, KX}})),
      X.d(), UX.p(), F.d());
  scale_axis(F.d(), sigd.d(), Da_ * KX * Ds, Dg, 1, 1, st);
  run(ST_TRIAD,
      G(modes({{Da_, GSg, KY * Ds * Dg}, {Ds * Dg, 1, 1}}), modes({{KY, 1, Ds * Dg}}),
        modes({{Gd, Ds * Dg, KY}})),
      Y.d(), UY.p(), Gt.d());
  // H[j0,kD,s,b] = sum_G D[b,j0,G,s] UD[G,kD]
  run(ST_TRIAD,
      G(modes({{D0, Gd * Ds, KD * Ds * Da_}, {Ds, 1, Da_}, {Da_, D0 * Gd * Ds, 1}}),
        modes({{KD, 1, Ds * Da_}}), modes({{Gd, Ds, KD}})),
      B.d(), UD.p(), H.d());
  X.release();
  Y.release();

  // ============================ squeezers (Eq. 5) ============================
  tm.mark(2);
  stage_prec(ST_SQUEEZE);
  std::vector<DMat> Ms(d - 1), Nts(d - 1);  // M[(a,b),k] and N^T[(a,b),k]
  std::vector<int64_t> Kn(d - 1, 0);
  spec_sq.assign(d - 1, {});
  {
    DevBuf om_d(Da_ * Da_ * sizeof(double), st), om_y(Dg * Dg * sizeof(double), st),
        om_a(Da_ * Da_ * sizeof(double), st), om_x(Dg * Dg * sizeof(double), st);
    const int64_t JKS = D0 * KD * Ds, IKS = D0 * KA * Ds;
    run(ST_SQUEEZE, G(modes({{Da_, 1, Da_}}), modes({{Da_, 1, 1}}), modes({{JKS, Da_, Da_}})), H.d(), H.d(), om_d.d());
    run(ST_SQUEEZE, G(modes({{Da_, 1, Da_}}), modes({{Da_, 1, 1}}), modes({{IKS, Da_, Da_}})), E.d(), E.d(), om_a.d());
    {
      const int64_t KSg = KY * Ds * Dg;
      DevBuf t(Da_ * KSg * sizeof(double), st);
      run(ST_SQUEEZE, G(modes({{Da_, 1, KSg}}), modes({{KSg, 1, 1}}), modes({{Da_, Da_, KSg}})), om_d.d(), Gt.d(), t.d());
      run(ST_SQUEEZE, G(modes({{Dg, 1, Dg}}), modes({{Dg, 1, 1}}), modes({{Da_ * KY * Ds, Dg, Dg}})), t.d(), Gt.d(), om_y.d());
    }
    {
      const int64_t KSg = KX * Ds * Dg;
      DevBuf t(Da_ * KSg * sizeof(double), st);
      run(ST_SQUEEZE, G(modes({{Da_, 1, KSg}}), modes({{KSg, 1, 1}}), modes({{Da_, Da_, KSg}})), om_a.d(), F.d(), t.d());
      run(ST_SQUEEZE, G(modes({{Dg, 1, Dg}}), modes({{Dg, 1, 1}}), modes({{Da_ * KX * Ds, Dg, Dg}})), t.d(), F.d(), om_x.d());
    }
    // Fy[a,kX,s,g'] = sum_g F[..,g] Om_Y[g,g'];  Gx likewise with Om_X
    DevBuf Fy(Da_ * KX * Ds * Dg * sizeof(double), st), Gx(Da_ * KY * Ds * Dg * sizeof(double), st);
    run(ST_SQUEEZE, G(modes({{Da_ * KX * Ds, Dg, Dg}}), modes({{Dg, 1, 1}}), modes({{Dg, 1, Dg}})), F.d(), om_y.d(), Fy.d());
    run(ST_SQUEEZE, G(modes({{Da_ * KY * Ds, Dg, Dg}}), modes({{Dg, 1, 1}}), modes({{Dg, 1, Dg}})), Gt.d(), om_x.d(), Gx.d());

    const int64_t P = Ds * Ds;
    std::vector<DevBuf> rhoL(d - 1), rhoR(d - 1);
    // separate leg (position d-1)
    {
      DevBuf eps(Ds * Da_ * Ds * Da_ * sizeof(double), st), phi(Da_ * Ds * Da_ * Ds * sizeof(double), st);
      run(ST_SQUEEZE, G(modes({{Ds * Da_, 1, Ds * Da_}}), modes({{Ds * Da_, 1, 1}}), modes({{D0 * KA, Ds * Da_, Ds * Da_}})),
          E.d(), E.d(), eps.d());
      run(ST_SQUEEZE,
          G(modes({{Da_, KX * Ds * Dg, Ds * Da_ * Ds}, {Ds, Dg, Da_ * Ds}}),
            modes({{Da_, KX * Ds * Dg, Ds}, {Ds, Dg, 1}}), modes({{KX, Ds * Dg, Ds * Dg}, {Dg, 1, 1}})),
          Fy.d(), F.d(), phi.d());
      rhoL[d - 2] = DevBuf(P * P * sizeof(double), st);
      run(ST_SQUEEZE,
          G(modes({{Ds, Da_ * Ds * Da_, Ds * Ds * Ds}, {Ds, Da_, Ds}}),
            modes({{Ds, Da_ * Ds, Ds * Ds}, {Ds, 1, 1}}),
            modes({{Da_, Ds * Da_, Ds * Da_ * Ds}, {Da_, 1, Ds}})),
          eps.d(), phi.d(), rhoL[d - 2].d());
      DevBuf gam(Da_ * Ds * Da_ * Ds * sizeof(double), st), eta(Ds * Da_ * Ds * Da_ * sizeof(double), st);
      run(ST_SQUEEZE,
          G(modes({{Da_, KY * Ds * Dg, Ds * Da_ * Ds}, {Ds, Dg, Da_ * Ds}}),
            modes({{Da_, KY * Ds * Dg, Ds}, {Ds, Dg, 1}}), modes({{KY, Ds * Dg, Ds * Dg}, {Dg, 1, 1}})),
          Gx.d(), Gt.d(), gam.d());
      run(ST_SQUEEZE, G(modes({{Ds * Da_, 1, Ds * Da_}}), modes({{Ds * Da_, 1, 1}}), modes({{D0 * KD, Ds * Da_, Ds * Da_}})),
          H.d(), H.d(), eta.d());
      rhoR[d - 2] = DevBuf(P * P * sizeof(double), st);
      // rho_R[(a,b),(a',b')] = sum_{b,b'} gam[be,a,be',a'] eta[b,be,b',be']
      run(ST_SQUEEZE,
          G(modes({{Ds, Da_ * Ds, Ds * Ds * Ds}, {Ds, 1, Ds}}),
            modes({{Ds, Da_ * Ds * Da_, Ds * Ds}, {Ds, Da_, 1}}),
            modes({{Da_, Ds * Da_ * Ds, Ds * Da_}, {Da_, Ds, 1}})),
          gam.d(), eta.d(), rhoR[d - 2].d());
    }
    if (g > 0) {
      // Env_L[kA,kA',kX,kX'] = sum_{a,a'} P_E[kA,kA',a,a'] P_F[a,a',kX,kX']
      DevBuf pe(KA * KA * Da_ * Da_ * sizeof(double), st), pf(Da_ * Da_ * KX * KX * sizeof(double), st);
      run(ST_SQUEEZE,
          G(modes({{KA, Ds * Da_, KA * Da_ * Da_}, {Da_, 1, Da_}}), modes({{KA, Ds * Da_, Da_ * Da_}, {Da_, 1, 1}}),
            modes({{D0, KA * Ds * Da_, KA * Ds * Da_}, {Ds, Da_, Da_}})),
          E.d(), E.d(), pe.d());
      run(ST_SQUEEZE,
          G(modes({{Da_, KX * Ds * Dg, Da_ * KX * KX}, {KX, Ds * Dg, KX}}),
            modes({{Da_, KX * Ds * Dg, KX * KX}, {KX, Ds * Dg, 1}}), modes({{Ds * Dg, 1, 1}})),
          Fy.d(), F.d(), pf.d());
      DevBuf envL(KA * KA * KX * KX * sizeof(double), st);
      run(ST_SQUEEZE, G(modes({{KA * KA, Da_ * Da_, KX * KX}}), modes({{KX * KX, 1, 1}}), modes({{Da_ * Da_, 1, KX * KX}})),
          pe.d(), pf.d(), envL.d());
      DevBuf pg(KY * KY * Da_ * Da_ * sizeof(double), st), ph(Da_ * Da_ * KD * KD * sizeof(double), st);
      run(ST_SQUEEZE,
          G(modes({{KY, Ds * Dg, KY * Da_ * Da_}, {Da_, KY * Ds * Dg, Da_}}),
            modes({{KY, Ds * Dg, Da_ * Da_}, {Da_, KY * Ds * Dg, 1}}), modes({{Ds * Dg, 1, 1}})),
          Gx.d(), Gt.d(), pg.d());
      run(ST_SQUEEZE,
          G(modes({{Da_, 1, Da_ * KD * KD}, {KD, Ds * Da_, KD}}), modes({{Da_, 1, KD * KD}, {KD, Ds * Da_, 1}}),
            modes({{D0, KD * Ds * Da_, KD * Ds * Da_}, {Ds, Da_, Da_}})),
          H.d(), H.d(), ph.d());
      DevBuf envR(KY * KY * KD * KD * sizeof(double), st);
      run(ST_SQUEEZE, G(modes({{KY * KY, Da_ * Da_, KD * KD}}), modes({{KD * KD, 1, 1}}), modes({{Da_ * Da_, 1, KD * KD}})),
          pg.d(), ph.d(), envR.d());
      for (int nu = 1; nu <= g; ++nu) {
        const int64_t Dn = D[nu];
        const int64_t Dz = Gd / Dn;  // product of the other group legs (1 when g == 1)
        // stride of leg nu and of the others inside the group index (row-major group legs)
        const int64_t snu = prod(D, nu + 1, 1 + g);
        auto pairgram = [&](const DMat& U, int64_t K, DevBuf& out) {
          out = DevBuf(Dn * Dn * K * K * sizeof(double), st);
          // out[a,a',k,k'] = sum_z U[(..a..z..),k] U[(..a'..z..),k']
          ModeIdx kz;
          if (g == 1) kz = modes({});
          else if (nu == 1) kz = modes({{Dz, K, K}});        // z = leg 2, stride K
          else kz = modes({{Dz, Dn * K, Dn * K}});           // z = leg 1, stride D2*K
          run(ST_SQUEEZE,
              G(modes({{Dn, snu * K, Dn * K * K}, {K, 1, K}}), modes({{Dn, snu * K, K * K}, {K, 1, 1}}), kz),
              U.p(), U.p(), out.d());
        };
        DevBuf ii, jj, kk, ll;
        pairgram(UA, KA, ii);
        pairgram(UX, KX, jj);
        pairgram(UY, KY, kk);
        pairgram(UD, KD, ll);
        const int64_t Pn = Dn * Dn;
        DevBuf t(Pn * KX * KX * sizeof(double), st);
        run(ST_SQUEEZE, G(modes({{Pn, KA * KA, KX * KX}}), modes({{KX * KX, 1, 1}}), modes({{KA * KA, 1, KX * KX}})),
            ii.d(), envL.d(), t.d());
        rhoL[nu - 1] = DevBuf(Pn * Pn * sizeof(double), st);
        run(ST_SQUEEZE,
            G(modes({{Dn, Dn * KX * KX, Dn * Dn * Dn}, {Dn, KX * KX, Dn}}),
              modes({{Dn, Dn * KX * KX, Dn * Dn}, {Dn, KX * KX, 1}}), modes({{KX * KX, 1, 1}})),
            t.d(), jj.d(), rhoL[nu - 1].d());
        DevBuf t2(Pn * KD * KD * sizeof(double), st);
        run(ST_SQUEEZE, G(modes({{Pn, KY * KY, KD * KD}}), modes({{KD * KD, 1, 1}}), modes({{KY * KY, 1, KD * KD}})),
            kk.d(), envR.d(), t2.d());
        rhoR[nu - 1] = DevBuf(Pn * Pn * sizeof(double), st);
        run(ST_SQUEEZE,
            G(modes({{Dn, Dn * KD * KD, Dn * Dn * Dn}, {Dn, KD * KD, Dn}}),
              modes({{Dn, Dn * KD * KD, Dn * Dn}, {Dn, KD * KD, 1}}), modes({{KD * KD, 1, 1}})),
            t2.d(), ll.d(), rhoR[nu - 1].d());
      }
    }
    // oblique projectors: C = R_L R_R^T = U S V^T, M = R_R^T V_k S^-1/2, N = S^-1/2 U_k^T R_L
    for (int nu = 1; nu <= d - 1; ++nu) {
      const int64_t Dn = D[nu], Pn = Dn * Dn;
      DMat RtL, RtR;
      factor(rhoL[nu - 1].d(), Pn, KIND_SQ_LEFT + nu - 1, RtL);
      factor(rhoR[nu - 1].d(), Pn, KIND_SQ_RIGHT + nu - 1, RtR);
      const int64_t kL = RtL.cols, kR = RtR.cols;
      DevBuf C(kL * kR * sizeof(double), st);
      eng.mm(kL, kR, Pn, RtL.p(), kL, true, RtR.p(), kR, false, C.d(), kR);
      SvdResult cs = eng.svd(C.d(), kL, kR);
      const int64_t k = multiplet_cut(cs.s, keep_count(cs.s, 1e-12, chi()), tau);
      TATRG_CHECK(k >= 1, TATRG_ENUMERIC, "squeezer core is zero");
      spec_sq[nu - 1] = cs.s;
      DevBuf isq(k * sizeof(double), st);
      {
        std::vector<double> v(cs.s.begin(), cs.s.begin() + k);
        for (auto& x : v) x = 1.0 / std::sqrt(x);
        TATRG_CUDA(cudaMemcpyAsync(isq.d(), v.data(), k * sizeof(double), cudaMemcpyHostToDevice, st));
      }
      Ms[nu - 1].buf = dalloc(Pn * k, st);
      Ms[nu - 1].rows = Pn;
      Ms[nu - 1].cols = k;
      Nts[nu - 1].buf = dalloc(Pn * k, st);
      Nts[nu - 1].rows = Pn;
      Nts[nu - 1].cols = k;
      eng.mm(Pn, k, kR, RtR.p(), kR, false, cs.V.p(), cs.V.cols, false, Ms[nu - 1].p(), k);
      eng.mm(Pn, k, kL, RtL.p(), kL, false, cs.U.p(), cs.U.cols, false, Nts[nu - 1].p(), k);
      scale_axis(Ms[nu - 1].p(), isq.d(), Pn, k, 1, 1, st);
      scale_axis(Nts[nu - 1].p(), isq.d(), Pn, k, 1, 1, st);
      canonical_cols(Ms[nu - 1].p(), Pn, int(k), cs.s, Nts[nu - 1].p(), Pn, false);
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
  DMat phi, psi;
  auto contract_side = [&](const DevBuf& E_, const DevBuf& F_, int64_t KA_, int64_t KX_, const DMat& I_,
                           const DMat& J_, const std::vector<DMat>& Ws, DMat& out) {
    // C1: em[i0,kA,a,b,k] = sum_a' E[i0,kA,a',a] W_sep[(a',b),k]
    DevBuf em(D0 * KA_ * Da_ * Ds * Ks * sizeof(double), st);
    run(ST_CONTRACT,
        G(modes({{D0 * KA_, Ds * Da_, Da_ * Ds * Ks}, {Da_, 1, Ds * Ks}}), modes({{Ds * Ks, 1, 1}}),
          modes({{Ds, Da_, Ds * Ks}})),
        E_.d(), Ws[d - 2].p(), em.d());
    // C2: q[i0,kA,k,kX,g] = sum_{a,b} em[i0,kA,a,b,k] F[a,kX,b,g]
    DevBuf qf(D0 * KA_ * Ks * KX_ * Dg * sizeof(double), st);
    run(ST_CONTRACT,
        G(modes({{D0 * KA_, Da_ * Ds * Ks, Ks * KX_ * Dg}, {Ks, 1, KX_ * Dg}}),
          modes({{KX_, Ds * Dg, Dg}, {Dg, 1, 1}}), modes({{Da_, Ds * Ks, KX_ * Ds * Dg}, {Ds, Ks, Dg}})),
        em.d(), F_.d(), qf.d());
    em.release();
    // C3: P[kA,kX,k_G] = sum I[a_G,kA] J[b_G,kX] prod_nu W_nu[(a_nu,b_nu),k_nu]
    DevBuf pm(KA_ * KX_ * Kg * sizeof(double), st);
    if (g == 0) {
      fill(pm.d(), 1, 1.0, st);
    } else if (g == 1) {
      const int64_t D1 = D[1], K1 = Kn[0];
      DevBuf t1(KA_ * D1 * K1 * sizeof(double), st);
      run(ST_CONTRACT, G(modes({{KA_, 1, D1 * K1}}), modes({{D1 * K1, 1, 1}}), modes({{D1, KA_, D1 * K1}})),
          I_.p(), Ws[0].p(), t1.d());
      run(ST_CONTRACT,
          G(modes({{KA_, D1 * K1, KX_ * K1}, {K1, 1, 1}}), modes({{KX_, 1, K1}}), modes({{D1, K1, KX_}})),
          t1.d(), J_.p(), pm.d());
    } else {
      const int64_t D1 = D[1], D2 = D[2], K1 = Kn[0], K2 = Kn[1];
      DevBuf t1(D2 * KA_ * D1 * K1 * sizeof(double), st), t2(KA_ * D1 * K1 * D2 * K2 * sizeof(double), st);
      run(ST_CONTRACT, G(modes({{D2 * KA_, 1, D1 * K1}}), modes({{D1 * K1, 1, 1}}), modes({{D1, D2 * KA_, D1 * K1}})),
          I_.p(), Ws[0].p(), t1.d());
      run(ST_CONTRACT,
          G(modes({{KA_ * D1 * K1, 1, D2 * K2}}), modes({{D2 * K2, 1, 1}}), modes({{D2, KA_ * D1 * K1, D2 * K2}})),
          t1.d(), Ws[1].p(), t2.d());
      run(ST_CONTRACT,
          G(modes({{KA_, D1 * K1 * D2 * K2, KX_ * K1 * K2}, {K1, D2 * K2, K2}, {K2, 1, 1}}),
            modes({{KX_, 1, K1 * K2}}), modes({{D1, K1 * D2 * K2, D2 * KX_}, {D2, K2, KX_}})),
          t2.d(), J_.p(), pm.d());
    }
    // C4: out[i0,k_G,k,g] = sum_{kA,kX} q[i0,kA,k,kX,g] P[kA,kX,k_G]
    out.buf = dalloc(rowsN * Dg, st);
    out.rows = rowsN;
    out.cols = Dg;
    run(ST_CONTRACT,
        G(modes({{D0, KA_ * Ks * KX_ * Dg, Kg * Ks * Dg}, {Ks, KX_ * Dg, Dg}, {Dg, 1, 1}}),
          modes({{Kg, 1, Ks * Dg}}), modes({{KA_, Ks * KX_ * Dg, KX_ * Kg}, {KX_, Dg, Kg}})),
        qf.d(), pm.d(), out.p());
  };
  contract_side(E, F, KA, KX, UA, UX, Ms, phi);
  // Psi: the same chain with H (for E), G (for F), L, K and the transposed N's; H carries
  // the backward leg j0(n) and L the group legs of site n, so (kD, kY) take the roles of
  // (kA, kX) with the pair order (a, b) = (leg at n+1^, leg at n) kept by N^T.
  {
    // hn[j0,kD,be,a,k] = sum_b H[j0,kD,b,be] N_sep[k,(a,b)]
    DevBuf hn(D0 * KD * Da_ * Ds * Ks * sizeof(double), st);
    run(ST_CONTRACT,
        G(modes({{D0 * KD, Ds * Da_, Da_ * Ds * Ks}, {Da_, 1, Ds * Ks}}), modes({{Ds, Ds * Ks, Ks}, {Ks, 1, 1}}),
          modes({{Ds, Da_, Ks}})),
        H.d(), Nts[d - 2].p(), hn.d());
    DevBuf qp(D0 * KD * Ks * KY * Dg * sizeof(double), st);
    run(ST_CONTRACT,
        G(modes({{D0 * KD, Da_ * Ds * Ks, Ks * KY * Dg}, {Ks, 1, KY * Dg}}),
          modes({{KY, Ds * Dg, Dg}, {Dg, 1, 1}}), modes({{Da_, Ds * Ks, KY * Ds * Dg}, {Ds, Ks, Dg}})),
        hn.d(), Gt.d(), qp.d());
    hn.release();
    // P'[kY,kD,k_G] = sum K[a_G,kY] L[b_G,kD] prod N_nu[k,(a,b)]
    DevBuf pm(KY * KD * Kg * sizeof(double), st);
    if (g == 0) {
      fill(pm.d(), 1, 1.0, st);
    } else if (g == 1) {
      const int64_t D1 = D[1], K1 = Kn[0];
      DevBuf t1(KY * D1 * K1 * sizeof(double), st);
      run(ST_CONTRACT, G(modes({{KY, 1, D1 * K1}}), modes({{D1 * K1, 1, 1}}), modes({{D1, KY, D1 * K1}})),
          UY.p(), Nts[0].p(), t1.d());
      run(ST_CONTRACT,
          G(modes({{KY, D1 * K1, KD * K1}, {K1, 1, 1}}), modes({{KD, 1, K1}}), modes({{D1, K1, KD}})),
          t1.d(), UD.p(), pm.d());
    } else {
      const int64_t D1 = D[1], D2 = D[2], K1 = Kn[0], K2 = Kn[1];
      DevBuf t1(D2 * KY * D1 * K1 * sizeof(double), st), t2(KY * D1 * K1 * D2 * K2 * sizeof(double), st);
      run(ST_CONTRACT, G(modes({{D2 * KY, 1, D1 * K1}}), modes({{D1 * K1, 1, 1}}), modes({{D1, D2 * KY, D1 * K1}})),
          UY.p(), Nts[0].p(), t1.d());
      run(ST_CONTRACT,
          G(modes({{KY * D1 * K1, 1, D2 * K2}}), modes({{D2 * K2, 1, 1}}), modes({{D2, KY * D1 * K1, D2 * K2}})),
          t1.d(), Nts[1].p(), t2.d());
      run(ST_CONTRACT,
          G(modes({{KY, D1 * K1 * D2 * K2, KD * K1 * K2}, {K1, D2 * K2, K2}, {K2, 1, 1}}),
            modes({{KD, 1, K1 * K2}}), modes({{D1, K1 * D2 * K2, D2 * KD}, {D2, K2, KD}})),
          t2.d(), UD.p(), pm.d());
    }
    // Psi[j0,k_G,k,g] = sum_{kD,kY} qp[j0,kD,k,kY,g] P'[kY,kD,k_G]
    psi.buf = dalloc(rowsN * Dg, st);
    psi.rows = rowsN;
    psi.cols = Dg;
    run(ST_CONTRACT,
        G(modes({{D0, KD * Ks * KY * Dg, Kg * Ks * Dg}, {Ks, KY * Dg, Dg}, {Dg, 1, 1}}),
          modes({{Kg, 1, Ks * Dg}}), modes({{KD, Ks * KY * Dg, Kg}, {KY, Dg, KD * Kg}})),
        qp.d(), pm.d(), psi.p());
  }
  E.release();
  F.release();
  Gt.release();
  H.release();

  // ============================ re-split and rotation ============================
  tm.mark(4);
  stage_prec(ST_RESPLIT);
  std::vector<int64_t> newD(d);
  newD[0] = D0;
  for (int nu = 1; nu < d; ++nu) newD[nu] = Kn[nu - 1];
  resplit_and_rotate(phi, psi, rowsN, Dg, newD);
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
  info.kernel_launches = int(eng.stats().launches - launches0);
  info.tc_launches = int(eng.stats().tc_launches - tc0);
  info.tc_flops = eng.stats().flops_tc - tcf0;
  info.tc_ms = eng.stats().drain_ms();
}

void tatrg_ctx::resplit_and_rotate(DMat& phi, DMat& psi, int64_t rows, int64_t Dg,
                                   const std::vector<int64_t>& newD) {
  cudaStream_t st = stream;
  flops[ST_RESPLIT] += 8.0 * double(rows) * double(Dg) * double(Dg);
  OrthResult qa = eng.orth(phi.p(), rows, Dg);
  OrthResult qb = eng.orth(psi.p(), rows, Dg);
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
  eng.gemm(G(modes({{D0, Kr * ka, Dn}, {Kr, ka, D0 * Dn}}), modes({{Dn, 1, 1}}), modes({{ka, 1, cs.U.cols}})),
           qa.Q.p(), cs.U.p(), An.d());
  // B'[a, rot] = (Q_Psi V_k)^T
  eng.gemm(G(modes({{D0, Kr * kb, 1}, {Kr, kb, D0}}), modes({{Dn, 1, rows}}), modes({{kb, 1, cs.V.cols}})),
           qb.Q.p(), cs.V.p(), Bn.d());
  canonical_cols(An.d(), rows, int(Dn), cs.s, Bn.d(), rows, true);
  A = std::move(An);
  B = std::move(Bn);
  Da = Dn;
  s.assign(cs.s.begin(), cs.s.begin() + Dn);
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
    TATRG_CHECK(params->precision >= TATRG_FP64 && params->precision <= TATRG_BF16X3, TATRG_EINVAL,
                "tatrg_create: unknown precision");
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

tatrg_status tatrg_grad(tatrg_ctx* ctx, double*, double*, double*) {
  if (!ctx) return TATRG_EINVAL;
  ctx->err = "tatrg_grad: adjoint kernels are not built in this version";
  return TATRG_ENOTIMPL;
}

tatrg_status tatrg_sweep(tatrg_ctx* ctx, const double* betas, int nbeta, double h, int d,
                         int nsteps, double* lnZ_out) {
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
    std::mutex mu;
    tatrg_status first = TATRG_OK;
    std::string first_msg;
    auto fail = [&](tatrg_status c, const std::string& m) {
      std::lock_guard<std::mutex> l(mu);
      if (first == TATRG_OK) { first = c; first_msg = m; }
    };
    std::vector<std::thread> pool;
    for (int w = 0; w < nw; ++w) {
      pool.emplace_back([&]() {
        cudaStream_t s = nullptr;
        try {
          TATRG_CUDA(cudaSetDevice(dev));
          TATRG_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
          for (int i = next++; i < nbeta && first == TATRG_OK; i = next++) {
            tatrg_ctx sub(ctx->p, s);
            sub.replica = uint32_t(i);
            sub.init_ising(betas[i], h, d);
            for (int k = 0; k < nsteps; ++k) sub.rg_step();
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

tatrg_status tatrg_spectrum(const tatrg_ctx* ctx, int kind, double* out, int* n) {
  if (!ctx || !n) return TATRG_EINVAL;
  const std::vector<double>* v = nullptr;
  if (kind == 0) v = &ctx->spec_s;
  else if (kind == 1) v = &ctx->spec_sigma;
  else if (kind >= 2 && size_t(kind - 2) < ctx->spec_sq.size()) v = &ctx->spec_sq[kind - 2];
  if (!v) return TATRG_EINVAL;
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
    ctx->d = d;
    ctx->D.assign(dims, dims + d);
    ctx->Da = dims[d];
    const int64_t F = prod(ctx->D, 0, ctx->D.size());
    ctx->A = DevBuf(F * ctx->Da * sizeof(double), ctx->stream);
    ctx->B = DevBuf(F * ctx->Da * sizeof(double), ctx->stream);
    TATRG_CUDA(cudaMemcpyAsync(ctx->A.d(), A, F * ctx->Da * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    TATRG_CUDA(cudaMemcpyAsync(ctx->B.d(), B, F * ctx->Da * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    ctx->s.assign(s, s + ctx->Da);
    ctx->upload_s();
    ctx->step = step;
    // keep ln c_k so that partial_lnz() reproduces the given sum: put it all in k = 0
    ctx->lnc.assign(step + 1, 0.0);
    ctx->lnc[0] = partial_lnz;
    ctx->ready = true;
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

tatrg_status tatrg_contract(const tatrg_contraction* c, int precision, const double* A, const double* B,
                            double* C, void* stream) {
  return guard(nullptr, [&] {
    TATRG_CHECK(c && A && B && C, TATRG_EINVAL, "tatrg_contract: null argument");
    TATRG_CHECK(precision >= 0 && precision <= 2, TATRG_EINVAL, "tatrg_contract: bad precision");
    GemmDesc g;
    g.m = modes({{c->m_ext[0], c->m_sA[0], c->m_sC[0]}, {c->m_ext[1], c->m_sA[1], c->m_sC[1]},
                 {c->m_ext[2], c->m_sA[2], c->m_sC[2]}, {c->m_ext[3], c->m_sA[3], c->m_sC[3]}});
    g.n = modes({{c->n_ext[0], c->n_sB[0], c->n_sC[0]}, {c->n_ext[1], c->n_sB[1], c->n_sC[1]},
                 {c->n_ext[2], c->n_sB[2], c->n_sC[2]}, {c->n_ext[3], c->n_sB[3], c->n_sC[3]}});
    g.k = modes({{c->k_ext[0], c->k_sA[0], c->k_sB[0]}, {c->k_ext[1], c->k_sA[1], c->k_sB[1]},
                 {c->k_ext[2], c->k_sA[2], c->k_sB[2]}, {c->k_ext[3], c->k_sA[3], c->k_sB[3]}});
    for (int i = 0; i < 4; ++i)
      TATRG_CHECK(c->m_ext[i] >= 1 && c->n_ext[i] >= 1 && c->k_ext[i] >= 1, TATRG_EINVAL,
                  "tatrg_contract: extents must be >= 1");
    g.alpha = c->alpha;
    g.beta = c->beta;
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

}  // extern "C"
