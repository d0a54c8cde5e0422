// FP64 CUDA-core kernels: the multi-mode contraction (GEMM) used by the FP64 form and
// for small contractions in every form, the Philox Gaussian sketch, and the elementwise
// and reduction helpers of the RG step.
#include "kernels.cuh"
#include "philox.cuh"

namespace tatrg {

// ---------------------------------------------------------------------------------
// Multi-mode FP64 GEMM.  64x64 output tile, K tile of 16, 256 threads with a 4x4
// register tile each; operand offsets for the tile's rows / columns / k slice are
// decomposed once into shared memory, so arbitrary mode strides cost one table lookup
// per element load.  gridDim.z splits K; each split writes its partial tile to a workspace
// and a second kernel adds the splits in order, so results do not depend on scheduling.
namespace {
constexpr int BM = 64, BN = 64, BK = 16;

struct GemmArgs {
  DevModes m, n, k;  // m: (A, C) strides, n: (B, C) strides, k: (A, B) strides
  int64_t M, N, K, kchunk;
  double alpha, beta;
  int a_mcontig, b_ncontig;  // 1: stride-1 mode is m (for A) / n (for B)
  int split;
  const double* A;
  const double* B;
  double* C;
  double* W;  // split > 1: split x M x N row-major partials
};

__global__ void __launch_bounds__(256) gemm_f64_kernel(GemmArgs g) {
  __shared__ double As[2][BK][BM + 1];
  __shared__ double Bs[2][BK][BN + 1];
  __shared__ int64_t offAm[BM], offCm[BM], offBn[BN], offCn[BN];
  __shared__ int64_t offAk[2][BK], offBk[2][BK];

  const int tid = threadIdx.x;
  const int64_t m0 = int64_t(blockIdx.x) * BM;
  const int64_t n0 = int64_t(blockIdx.y) * BN;
  const int64_t kbeg = int64_t(blockIdx.z) * g.kchunk;
  const int64_t kend = min(g.K, kbeg + g.kchunk);

  if (tid < BM) {
    int64_t mm = m0 + tid;
    int64_t a = 0, c = 0;
    if (mm < g.M) mode_offsets(g.m, mm, a, c);
    offAm[tid] = a;
    offCm[tid] = c;
  } else if (tid < BM + BN) {
    int t = tid - BM;
    int64_t nn = n0 + t;
    int64_t b = 0, c = 0;
    if (nn < g.N) mode_offsets(g.n, nn, b, c);
    offBn[t] = b;
    offCn[t] = c;
  }
  auto koffsets = [&](int buf, int64_t kt) {
    if (tid < BK) {
      int64_t kk = kt + tid;
      int64_t a = 0, b = 0;
      if (kk < kend) mode_offsets(g.k, kk, a, b);
      offAk[buf][tid] = a;
      offBk[buf][tid] = b;
    }
  };
  koffsets(0, kbeg);
  __syncthreads();

  double ra[4], rb[4];
  auto load = [&](int buf, int64_t kt) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int e = tid + 256 * i;
      int mm, kk;
      if (g.a_mcontig) { mm = e % BM; kk = e / BM; } else { kk = e % BK; mm = e / BK; }
      double v = 0.0;
      if (m0 + mm < g.M && kt + kk < kend) v = g.A[offAm[mm] + offAk[buf][kk]];
      ra[i] = v;
      int nn;
      if (g.b_ncontig) { nn = e % BN; kk = e / BN; } else { kk = e % BK; nn = e / BK; }
      double w = 0.0;
      if (n0 + nn < g.N && kt + kk < kend) w = g.B[offBn[nn] + offBk[buf][kk]];
      rb[i] = w;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int e = tid + 256 * i;
      int mm, kk;
      if (g.a_mcontig) { mm = e % BM; kk = e / BM; } else { kk = e % BK; mm = e / BK; }
      As[buf][kk][mm] = ra[i];
      int nn;
      if (g.b_ncontig) { nn = e % BN; kk = e / BN; } else { kk = e % BK; nn = e / BK; }
      Bs[buf][kk][nn] = rb[i];
    }
  };

  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  const int tx = tid % 16, ty = tid / 16;
  int buf = 0;
  load(0, kbeg);
  store(0);
  __syncthreads();
  for (int64_t kt = kbeg; kt < kend; kt += BK) {
    const bool more = kt + BK < kend;
    if (more) {
      koffsets(buf ^ 1, kt + BK);
      __syncthreads();
      load(buf ^ 1, kt + BK);
    }
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[buf][kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[buf][kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    if (more) {
      store(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  }

#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int mm = ty + 16 * i;
    if (m0 + mm >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int nn = tx + 16 * j;
      if (n0 + nn >= g.N) continue;
      if (g.split > 1) {
        g.W[(int64_t(blockIdx.z) * g.M + m0 + mm) * g.N + n0 + nn] = acc[i][j];
      } else {
        double* c = g.C + offCm[mm] + offCn[nn];
        double v = g.alpha * acc[i][j];
        if (g.beta != 0.0) v += g.beta * *c;
        *c = v;
      }
    }
  }
}

// C[m, n] = alpha * sum_z W[z, m, n] (z in order) + beta * C[m, n], C through its modes
__global__ void split_reduce_kernel(const double* W, int split, double* C, DevModes m, DevModes n,
                                    int64_t M, int64_t N, double alpha, double beta) {
  const int64_t total = M * N;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = e / N, j = e - (e / N) * N;
    double acc = 0.0;
    for (int z = 0; z < split; ++z) acc += W[int64_t(z) * total + e];
    int64_t a, c, b, d;
    mode_offsets(m, i, a, c);
    mode_offsets(n, j, b, d);
    double* p = C + c + d;
    double v = alpha * acc;
    if (beta != 0.0) v += beta * *p;
    *p = v;
  }
}

__global__ void scale_modes_kernel(double* C, DevModes m, DevModes n, int64_t M, int64_t N,
                                   double beta) {
  int64_t total = M * N;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    int64_t i = e / N, j = e - (e / N) * N;
    int64_t a, c, b, d;
    mode_offsets(m, i, a, c);
    mode_offsets(n, j, b, d);
    double* p = C + c + d;
    *p = beta == 0.0 ? 0.0 : beta * *p;
  }
}

int stride1_first(const ModeIdx& x, bool first) {
  // 1 when the innermost mode has unit stride in the chosen operand
  if (x.n == 0) return 0;
  return (first ? x.s0[x.n - 1] : x.s1[x.n - 1]) == 1 ? 1 : 0;
}
}  // namespace

void gemm_f64(const GemmDesc& d0, const double* A, const double* B, double* C, cudaStream_t s,
              Stats* st) {
  if (d0.m.total() == 0 || d0.n.total() == 0) return;
  check_gemm(d0, A, B, C);
  GemmDesc d = d0;
  if (cdiv(d0.n.total(), BN) > cdiv(d0.m.total(), BM)) {
    // C^T = B^T A^T: the longer output dimension goes on grid.x
    d.m = d0.n;
    d.n = d0.m;
    for (int i = 0; i < kMaxModes; ++i) std::swap(d.k.s0[i], d.k.s1[i]);
    std::swap(A, B);
  }
  const int64_t M = d.m.total(), N = d.n.total(), K = d.k.total();
  GemmArgs g;
  g.m = dev(d.m);
  g.n = dev(d.n);
  g.k = dev(d.k);
  g.M = M;
  g.N = N;
  g.K = K;
  g.alpha = d.alpha;
  g.beta = d.beta;
  g.A = A;
  g.B = B;
  g.C = C;
  g.a_mcontig = stride1_first(d.m, true) && !stride1_first(d.k, true);
  g.b_ncontig = stride1_first(d.n, true) && !stride1_first(d.k, false);
  const int64_t tiles = cdiv(M, BM) * cdiv(N, BN);
  int split = 1;
  const int64_t target = 4 * int64_t(sm_count());
  if (tiles < target && K > 4 * BK) {
    split = int(std::min<int64_t>(cdiv(target, tiles), cdiv(K, 4 * BK)));
    split = std::min(split, 1024);
  }
  int64_t kchunk = cdiv(cdiv(K, split), BK) * BK;
  split = int(cdiv(K, kchunk));
  if (K == 0) { split = 1; kchunk = 0; }
  g.split = split;
  g.kchunk = kchunk;
  g.W = nullptr;
  // C's offsets alone, for the kernels that address only C
  DevModes mc = dev(d.m), nc = dev(d.n);
  for (int i = 0; i < kMaxModes; ++i) { mc.s0[i] = mc.s1[i]; nc.s0[i] = nc.s1[i]; }
  const int rblocks = int(std::min<int64_t>(cdiv(M * N, 256), 4096));
  if (K == 0) {
    scale_modes_kernel<<<rblocks, 256, 0, s>>>(C, mc, nc, M, N, d.beta);
    TATRG_CUDA(cudaGetLastError());
    if (st) st->launches++;
    return;
  }
  DevBuf work;
  if (split > 1) {
    work.alloc(size_t(split) * size_t(M) * size_t(N) * sizeof(double), s);
    g.W = work.d();
  }
  dim3 grid(unsigned(cdiv(M, BM)), unsigned(cdiv(N, BN)), unsigned(split));
  TATRG_CHECK(grid.y <= 65535 && cdiv(M, BM) < (int64_t(1) << 31), TATRG_EINVAL,
              "gemm_f64: problem too large for the grid");
  gemm_f64_kernel<<<grid, 256, 0, s>>>(g);
  TATRG_CUDA(cudaGetLastError());
  if (split > 1) {
    split_reduce_kernel<<<rblocks, 256, 0, s>>>(g.W, split, C, mc, nc, M, N, d.alpha, d.beta);
    TATRG_CUDA(cudaGetLastError());
    if (st) st->launches++;
  }
  if (st) {
    st->launches++;
    st->flops_f64 += 2.0 * double(M) * double(N) * double(K);
  }
}

// ---------------------------------------------------------------------------------
// Philox4x32-10 + Box-Muller (philox.cuh).  One thread per output pair.
namespace {
__global__ void gaussian_kernel(uint64_t seed, uint32_t sid, uint32_t replica, int64_t n,
                                double* out) {
  const int64_t npairs = (n + 1) / 2;
  for (int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; p < npairs;
       p += int64_t(gridDim.x) * blockDim.x) {
    uint32_t w[4];
    philox4x32_10(seed, sid, replica, p, w);
    double u1 = u53(w[0], w[1]), u2 = u53(w[2], w[3]);
    double rad = sqrt(-2.0 * log(u1));
    double ang = 2.0 * 3.141592653589793 * u2;
    out[2 * p] = rad * cos(ang);
    if (2 * p + 1 < n) out[2 * p + 1] = rad * sin(ang);
  }
}

// The same stream with Box-Muller in float arithmetic (gauss_pair_f32).
__global__ void gaussian_f32_kernel(uint64_t seed, uint32_t sid, uint32_t replica, int64_t n,
                                    double* out) {
  const int64_t npairs = (n + 1) / 2;
  for (int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; p < npairs;
       p += int64_t(gridDim.x) * blockDim.x) {
    float z0, z1;
    gauss_pair_f32(seed, sid, replica, p, z0, z1);
    if (2 * p + 1 < n) {
      reinterpret_cast<double2*>(out)[p] = make_double2(double(z0), double(z1));
    } else {
      out[2 * p] = double(z0);
    }
  }
}
}  // namespace

namespace {
__global__ void philox_words_kernel(uint64_t seed, uint32_t sid, uint32_t replica, uint64_t first,
                                    int64_t npairs, uint4* out) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < npairs;
       i += int64_t(gridDim.x) * blockDim.x) {
    uint32_t w[4];
    philox4x32_10(seed, sid, replica, int64_t(first + uint64_t(i)), w);  // counter modulo 2^64
    out[i] = make_uint4(w[0], w[1], w[2], w[3]);
  }
}
}  // namespace

void philox_words(uint64_t seed, uint32_t sid, uint32_t replica, uint64_t first, int64_t npairs,
                  uint32_t* out, cudaStream_t s) {
  TATRG_CHECK(out != nullptr && npairs >= 0, TATRG_EINVAL, "philox_words: bad argument");
  TATRG_CHECK((reinterpret_cast<uintptr_t>(out) & 15) == 0, TATRG_EINVAL,
              "philox_words: output must be 16-byte aligned");
  if (npairs == 0) return;
  check_extent(out, 4 * npairs - 1, sizeof(uint32_t), "philox_words");
  const int blocks = int(std::min<int64_t>(cdiv(npairs, 256), int64_t(sm_count()) * 32));
  philox_words_kernel<<<blocks, 256, 0, s>>>(seed, sid, replica, first, npairs, reinterpret_cast<uint4*>(out));
  TATRG_CUDA(cudaGetLastError());
}

void ensure_smem_attr(const void* fn, int bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, int> done;
  int dev = 0;
  TATRG_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> l(mu);
  auto key = std::make_pair(dev, fn);
  auto it = done.find(key);
  if (it != done.end() && it->second >= bytes) return;
  TATRG_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  done[key] = bytes;
}

int sm_count() {
  // per device ordinal: a process may drive several GPUs
  static std::mutex mu;
  static std::map<int, int> cache;
  int dev = 0;
  TATRG_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> l(mu);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  int n = 0;
  TATRG_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
  TATRG_CHECK(n >= 1, TATRG_ECUDA, "device reports no multiprocessors");
  cache[dev] = n;
  return n;
}

void gaussian(uint64_t seed, uint32_t sid, uint32_t replica, int64_t n, double* out,
              cudaStream_t s, bool float_math) {
  if (n <= 0) return;
  TATRG_CHECK(out != nullptr, TATRG_EINVAL, "gaussian: null output");
  check_extent(out, n - 1, sizeof(double), "gaussian");
  int64_t npairs = (n + 1) / 2;
  int blocks = int(std::min<int64_t>(cdiv(npairs, 256), int64_t(sm_count()) * 32));
  if (float_math) {
    TATRG_CHECK((reinterpret_cast<uintptr_t>(out) & 15) == 0, TATRG_EINVAL,
                "gaussian: output must be 16-byte aligned");
    gaussian_f32_kernel<<<blocks, 256, 0, s>>>(seed, sid, replica, n, out);
  } else {
    gaussian_kernel<<<blocks, 256, 0, s>>>(seed, sid, replica, n, out);
  }
  TATRG_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------------------------
// Elementwise helpers.
namespace {
__global__ void scale_axis_kernel(double* x, const double* v, int64_t outer, int64_t n,
                                  int64_t inner, int power) {
  int64_t total = outer * n * inner;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    int64_t i = (e / inner) % n;
    double w = v[i];
    if (power == 2) w = w * w;
    else if (power == -1) w = 1.0 / w;
    else if (power == -2) w = rsqrt(w);
    x[e] *= w;
  }
}

__global__ void copy_modes_kernel(double* dst, const double* src, DevModes m, int64_t total,
                                  double alpha) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    int64_t a, b;
    mode_offsets(m, e, a, b);
    dst[b] = alpha * src[a];
  }
}

__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85EBCA6Bu;
  h ^= h >> 13;
  h *= 0xC2B2AE35u;
  h ^= h >> 16;
  return h;
}

// Per-block partials of v[a] = sum_f w_f X[f, a] for row-major X (F x n) with
// w_f = (fmix32(f+1)+0.5)/2^32 - 0.5: block b takes rows [b*rows, (b+1)*rows), thread a
// adds its column in row order (consecutive threads read consecutive addresses).
__global__ void weighted_colsum_kernel(const double* X, int64_t F, int n, int64_t rows,
                                       double* part) {
  const int64_t f0 = int64_t(blockIdx.x) * rows, f1 = min(F, f0 + rows);
  for (int a = threadIdx.x; a < n; a += blockDim.x) {
    double acc = 0.0;
    for (int64_t f = f0; f < f1; ++f) {
      const double w = (double(fmix32(uint32_t(f + 1))) + 0.5) * (1.0 / 4294967296.0) - 0.5;
      acc = fma(w, X[f * n + a], acc);
    }
    part[int64_t(blockIdx.x) * n + a] = acc;
  }
}

// out[j] = sum_b part[b * width + j], b in order
__global__ void finish_partials_kernel(const double* part, int nb, int width, double* out) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < width; j += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int b = 0; b < nb; ++b) acc += part[int64_t(b) * width + j];
    out[j] = acc;
  }
}

// Sum of one value per thread over the block in a fixed order; the result is valid in
// thread 0.  red holds 32 doubles of shared memory.
__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < int(blockDim.x >> 5); ++w) t += red[w];
  return t;
}

// flip columns a of X (F x n, row-major) and rows a of Y (n x G) where v[a] < 0
__global__ void flip_kernel(double* X, int64_t F, int n, double* Y, int64_t G,
                            const double* v) {
  const int64_t tx = F * n, ty = (Y ? G * n : 0);
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < tx + ty;
       e += int64_t(gridDim.x) * blockDim.x) {
    if (e < tx) {
      int a = int(e % n);
      if (v[a] < 0.0) X[e] = -X[e];
    } else {
      int64_t e2 = e - tx;
      int a = int(e2 / G);
      if (v[a] < 0.0) Y[e2] = -Y[e2];
    }
  }
}

// Per-block partials of G[i, j] = sum_f X[f, a + i] w_j(f) for row-major X (F x n),
// i, j < m (m <= 32), with w_j(f) = (fmix32((f + 1) xor (j * 0x9E3779B9)) + 0.5) / 2^32 - 0.5.
// Block b takes rows [b*rows, (b+1)*rows); thread (i, j) adds in row order.
__global__ void multiplet_overlap_kernel(const double* X, int64_t F, int n, int a, int m,
                                         int64_t rows, double* part) {
  const int64_t f0 = int64_t(blockIdx.x) * rows, f1 = min(F, f0 + rows);
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
    const int i = t / m, j = t - (t / m) * m;
    double acc = 0.0;
    for (int64_t f = f0; f < f1; ++f) {
      const double w = (double(fmix32(uint32_t(f + 1) ^ (uint32_t(j) * 0x9E3779B9u))) + 0.5) *
                           (1.0 / 4294967296.0) - 0.5;
      acc = fma(X[f * n + a + i], w, acc);
    }
    part[int64_t(blockIdx.x) * m * m + t] = acc;
  }
}

// per-block partial sums of x (grid-stride, fixed order)
__global__ void sum_kernel(const double* x, int64_t n, double* part) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n;
       e += int64_t(gridDim.x) * blockDim.x)
    acc += x[e];
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// per-block partials of tTr = sum_a s_a sum_f A[f, a] B[a, f]
__global__ void trace_kernel(const double* A, const double* s, const double* B, int64_t F,
                             int Da, double* part) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < F * Da;
       e += int64_t(gridDim.x) * blockDim.x) {
    int64_t f = e / Da;
    int a = int(e - f * Da);
    acc += A[e] * s[a] * B[int64_t(a) * F + f];
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void ising_tensor_kernel(double beta, double h, int d, double* T) {
  const int n = 1 << (2 * d);
  double c = sqrt(2.0 * cosh(beta)), sn = sqrt(2.0 * sinh(beta));
  double w[2][2];
  w[0][0] = 0.5 * (c + sn);
  w[0][1] = 0.5 * (c - sn);
  w[1][0] = 0.5 * (c - sn);
  w[1][1] = 0.5 * (c + sn);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int si = 0; si < 2; ++si) {
      double t = exp(si == 0 ? h : -h);
      for (int leg = 0; leg < 2 * d; ++leg) {
        int x = (e >> (2 * d - 1 - leg)) & 1;
        t *= w[si][x];
      }
      acc += t;
    }
    T[e] = acc;
  }
}

__global__ void fill_kernel(double* x, int64_t n, double v) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n;
       e += int64_t(gridDim.x) * blockDim.x)
    x[e] = v;
}

__global__ void check_finite_kernel(const double* x, int64_t n, int* bad) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n;
       e += int64_t(gridDim.x) * blockDim.x)
    if (!isfinite(x[e])) { *bad = 1; return; }
}

int grid_for(int64_t n) { return int(std::max<int64_t>(1, std::min<int64_t>(cdiv(n, 256), int64_t(sm_count()) * 16))); }
}  // namespace

void scale_axis(double* x, const double* v, int64_t outer, int64_t n, int64_t inner, int power,
                cudaStream_t s) {
  int64_t total = outer * n * inner;
  if (total == 0) return;
  check_extent(x, total - 1, sizeof(double), "scale_axis");
  check_extent(v, n - 1, sizeof(double), "scale_axis weights");
  scale_axis_kernel<<<grid_for(total), 256, 0, s>>>(x, v, outer, n, inner, power);
  TATRG_CUDA(cudaGetLastError());
}

void copy_modes(double* dst, const double* src, const ModeIdx& m, double alpha, cudaStream_t s) {
  int64_t total = m.total();
  if (total == 0) return;
  check_extent(src, max_off0(m), sizeof(double), "copy_modes source");
  check_extent(dst, max_off1(m), sizeof(double), "copy_modes destination");
  copy_modes_kernel<<<grid_for(total), 256, 0, s>>>(dst, src, dev(m), total, alpha);
  TATRG_CUDA(cudaGetLastError());
}

namespace {
// rows per block for the row-chunked reductions: about 4 blocks per SM
int64_t row_chunk(int64_t F) { return std::max<int64_t>(64, cdiv(F, 4 * int64_t(sm_count()))); }

void finish_partials(const double* part, int nb, int width, double* out, cudaStream_t s) {
  finish_partials_kernel<<<int(cdiv(width, 256)), 256, 0, s>>>(part, nb, width, out);
  TATRG_CUDA(cudaGetLastError());
}
}  // namespace

void weighted_colsum(const double* X, int64_t F, int n, double* v, cudaStream_t s) {
  if (n == 0) return;
  if (F == 0) { fill(v, n, 0.0, s); return; }
  check_extent(X, F * n - 1, sizeof(double), "weighted_colsum");
  check_extent(v, n - 1, sizeof(double), "weighted_colsum output");
  const int64_t rows = row_chunk(F);
  const int nb = int(cdiv(F, rows));
  DevBuf part(size_t(nb) * n * sizeof(double), s);
  weighted_colsum_kernel<<<nb, std::min(256, 32 * int(cdiv(n, 32))), 0, s>>>(X, F, n, rows, part.d());
  TATRG_CUDA(cudaGetLastError());
  finish_partials(part.d(), nb, n, v, s);
}

void flip_by_sign(double* X, int64_t F, int n, double* Y, int64_t G, const double* v,
                  cudaStream_t s) {
  int64_t total = F * n + (Y ? G * n : 0);
  if (total == 0) return;
  check_extent(X, F * n - 1, sizeof(double), "flip_by_sign");
  if (Y) check_extent(Y, G * n - 1, sizeof(double), "flip_by_sign rows");
  flip_kernel<<<grid_for(total), 256, 0, s>>>(X, F, n, Y, G, v);
  TATRG_CUDA(cudaGetLastError());
}

void trace_asb(const double* A, const double* sv, const double* B, int64_t F, int Da,
               double* out, cudaStream_t s) {
  if (F * Da == 0) { fill(out, 1, 0.0, s); return; }
  check_extent(A, F * Da - 1, sizeof(double), "trace A");
  check_extent(B, F * Da - 1, sizeof(double), "trace B");
  const int nb = grid_for(F * Da);
  DevBuf part(size_t(nb) * sizeof(double), s);
  trace_kernel<<<nb, 256, 0, s>>>(A, sv, B, F, Da, part.d());
  TATRG_CUDA(cudaGetLastError());
  finish_partials(part.d(), nb, 1, out, s);
}

void multiplet_overlap(const double* X, int64_t F, int n, int a, int m, double* G, cudaStream_t s) {
  TATRG_CHECK(m >= 1 && m <= 32 && a >= 0 && a + m <= n, TATRG_EINVAL, "multiplet_overlap: bad block");
  check_extent(X, F * n - 1, sizeof(double), "multiplet_overlap");
  check_extent(G, int64_t(m) * m - 1, sizeof(double), "multiplet_overlap G");
  if (F == 0) { fill(G, int64_t(m) * m, 0.0, s); return; }
  const int64_t rows = row_chunk(F);
  const int nb = int(cdiv(F, rows));
  DevBuf part(size_t(nb) * m * m * sizeof(double), s);
  multiplet_overlap_kernel<<<nb, std::min(1024, 32 * int(cdiv(m * m, 32))), 0, s>>>(X, F, n, a, m, rows,
                                                                                  part.d());
  TATRG_CUDA(cudaGetLastError());
  finish_partials(part.d(), nb, m * m, G, s);
}

void sum_all(const double* x, int64_t n, double* out, cudaStream_t s) {
  if (n == 0) { fill(out, 1, 0.0, s); return; }
  check_extent(x, n - 1, sizeof(double), "sum_all");
  const int nb = grid_for(n);
  DevBuf part(size_t(nb) * sizeof(double), s);
  sum_kernel<<<nb, 256, 0, s>>>(x, n, part.d());
  TATRG_CUDA(cudaGetLastError());
  finish_partials(part.d(), nb, 1, out, s);
}

void ising_tensor(double beta, double h, int d, double* T, cudaStream_t s) {
  ising_tensor_kernel<<<grid_for(1 << (2 * d)), 256, 0, s>>>(beta, h, d, T);
  TATRG_CUDA(cudaGetLastError());
}

void fill(double* x, int64_t n, double v, cudaStream_t s) {
  if (n <= 0) return;
  check_extent(x, n - 1, sizeof(double), "fill");
  fill_kernel<<<grid_for(n), 256, 0, s>>>(x, n, v);
  TATRG_CUDA(cudaGetLastError());
}

void check_finite(const double* x, int64_t n, int* bad_dev, cudaStream_t s) {
  if (n <= 0) return;
  check_finite_kernel<<<grid_for(n), 256, 0, s>>>(x, n, bad_dev);
  TATRG_CUDA(cudaGetLastError());
}

}  // namespace tatrg
