// Small dense FP64 linear algebra: Cholesky (the core of CholeskyQR2; one block), the
// inverse of the triangular factor (one warp per column), and the one-sided (Hestenes)
// Jacobi SVD used for every core SVD / PSD eigenproblem of the RG step (swap core, triad
// Gram eigenvectors, squeezer factors and core, re-split): one block in shared memory for
// small problems, otherwise one cooperative grid with a block per column pair.

#include "kernels.cuh"


namespace tatrg {
namespace {

constexpr int kCholMaxN = 168;

// Right-looking Cholesky G + shift I = R^T R with the upper triangle of the working
// matrix in shared memory (full n x n storage, n <= kCholMaxN: 168^2 doubles and the
// kernel's own arrays fill the 227 KB a block may hold).  Step j scales row j by the
// pivot square root, then subtracts the outer product of the scaled row from the trailing
// block; the thread that updates the next diagonal entry takes its square root at once
// (FP64 square roots and divisions are scarce on this GPU, so they are not repeated per
// thread), which leaves two block barriers per step.  A pivot at or below 1e-14 of its
// original diagonal entry is a breakdown (status 1).
__global__ void __launch_bounds__(1024) cholesky_kernel(const double* G, int n, double* R,
                                                        int* status, double shift_rel) {
  extern __shared__ double W[];
  __shared__ double shift, djj_s[2];
  __shared__ int fail_s;
  __shared__ double red[32];
  __shared__ double ref[kCholMaxN];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int tx = tid & 31, ty = tid >> 5;  // 32 x 32 threads over (k, i)
  {
    double tr = 0.0;
    for (int i = tid; i < n; i += nt) tr += G[int64_t(i) * n + i];
    for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
    if (tx == 0) red[ty] = tr;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < (nt >> 5); ++w) t += red[w];
      shift = shift_rel * t;
      fail_s = 0;
    }
    __syncthreads();
  }
  const double sh = shift;
  for (int e = tid; e < n * n; e += nt) {
    const int i = e / n, k = e - (e / n) * n;
    W[e] = (k >= i) ? G[e] + (i == k ? sh : 0.0) : 0.0;
    if (i == k) ref[i] = G[e] + sh;
  }
  __syncthreads();
  // pivot j is checked and rooted by thread 0, which also updates entry (j, j) in step j - 1
  auto pivot = [&](int j) {
    const double d = W[j * n + j];
    if (!(d > 1e-14 * ref[j]) || !(ref[j] > 0.0)) fail_s = 1;
    else djj_s[j & 1] = sqrt(d);
  };
  if (tid == 0) pivot(0);
  for (int j = 0; j < n; ++j) {
    __syncthreads();
    if (fail_s) break;  // uniform across the block
    const double djj = djj_s[j & 1];
    for (int k = j + tid; k < n; k += nt) W[j * n + k] = (k == j) ? djj : W[j * n + k] / djj;
    __syncthreads();
    for (int i = j + 1 + ty; i < n; i += 32) {
      const double a = W[j * n + i];
      for (int k = i + ((tx - (i - (j + 1))) & 31); k < n; k += 32)
        W[i * n + k] = fma(-a, W[j * n + k], W[i * n + k]);
    }
    if (tid == 0 && j + 1 < n) pivot(j + 1);  // thread 0 updated entry (j + 1, j + 1) above
  }
  __syncthreads();
  const int fail = fail_s;
  for (int e = tid; e < n * n; e += nt) R[e] = fail ? 0.0 : W[e];
  if (tid == 0) *status = fail;
}

// Inverse of an upper-triangular matrix: column c of X = R^-1 is the back substitution
// R x = e_c, independent of the other columns, so one warp solves one column (x in the
// warp's slice of shared memory, the inner products split across lanes); no block-wide
// barrier is needed.  RS: the leading (cmax + 1) x (cmax + 1) block of R that the block's
// columns need is first copied to shared memory, so each back-substitution step reads
// shared memory instead of L2 (the same arithmetic in the same order).
template <bool RS>
__global__ void __launch_bounds__(128) tri_inverse_kernel(const double* R, int n, double* X) {
  extern __shared__ double xs[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int c = blockIdx.x * 4 + w;
  const int cmax = min(n - 1, blockIdx.x * 4 + 3);
  const int ld = RS ? cmax + 1 : n;
  const double* Rm = R;
  if (RS) {
    double* Rs = xs + 4 * n;
    for (int e = threadIdx.x; e < ld * ld; e += blockDim.x) {
      const int i = e / ld, k = e - (e / ld) * ld;
      Rs[e] = (k >= i) ? R[int64_t(i) * n + k] : 0.0;
    }
    __syncthreads();
    Rm = Rs;
  }
  if (c >= n) return;
  double* x = xs + w * n;
  for (int i = lane; i < n; i += 32) x[i] = 0.0;
  __syncwarp();
  for (int i = c; i >= 0; --i) {
    double acc = 0.0;
    for (int k = i + 1 + lane; k <= c; k += 32) acc += Rm[int64_t(i) * ld + k] * x[k];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) x[i] = ((i == c ? 1.0 : 0.0) - acc) / Rm[int64_t(i) * ld + i];
    __syncwarp();
  }
  for (int i = lane; i < n; i += 32) X[int64_t(i) * n + c] = x[i];
}

// One-sided Jacobi SVD.  Ac: column-major m x N workspace (N = n rounded up to even, the
// padding column is zero), Vc: column-major N x N initialised to the identity.  The m x N
// columns are worked on in shared memory and written back at the end; V stays in global
// memory (L2).
__global__ void __launch_bounds__(1024) jacobi_kernel(double* Acg, int64_t m, int N, double* Vc,
                                                      int max_sweeps, double tol, int* status) {
  extern __shared__ double Ac[];
  __shared__ int rotated;
  __shared__ double fro2, wsum[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t e = threadIdx.x; e < m * N; e += blockDim.x) Ac[e] = Acg[e];
  // Columns whose squared norm is below (4 eps)^2 ||A||_F^2 sit at the rounding floor:
  // they are treated as converged, otherwise rounding in a large-small pair keeps the
  // relative inner product above tol forever.
  __syncthreads();
  {
    double acc = 0.0;
    for (int64_t e = threadIdx.x; e < m * N; e += blockDim.x) acc = fma(Ac[e], Ac[e], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) wsum[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < nw; ++w) t += wsum[w];
      fro2 = t;
    }
  }
  __syncthreads();
  const double floor2 = 7.9e-31 * fro2;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int r = 0; r < N - 1; ++r) {
      for (int k = warp; k < N / 2; k += nw) {
        int p, q;
        if (k == 0) { p = N - 1; q = r % (N - 1); }
        else { p = (r + k) % (N - 1); q = (r + N - 1 - k) % (N - 1); }
        double* ap = Ac + int64_t(p) * m;
        double* aq = Ac + int64_t(q) * m;
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int64_t i = lane; i < m; i += 32) {
          double x = ap[i], y = aq[i];
          al = fma(x, x, al);
          be = fma(y, y, be);
          ga = fma(x, y, ga);
        }
        for (int o = 16; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        if (al > floor2 && be > floor2 && fabs(ga) > tol * sqrt(al) * sqrt(be)) {
          double zeta = (be - al) / (2.0 * ga);
          double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
          for (int64_t i = lane; i < m; i += 32) {
            double x = ap[i], y = aq[i];
            ap[i] = c * x - s * y;
            aq[i] = s * x + c * y;
          }
          double* vp = Vc + int64_t(p) * N;
          double* vq = Vc + int64_t(q) * N;
          for (int i = lane; i < N; i += 32) {
            double x = vp[i], y = vq[i];
            vp[i] = c * x - s * y;
            vq[i] = s * x + c * y;
          }
          if (lane == 0) rotated = 1;
        }
      }
      __syncthreads();
    }
    __syncthreads();
    if (!rotated) break;
    __syncthreads();
  }
  for (int64_t e = threadIdx.x; e < m * N; e += blockDim.x) Acg[e] = Ac[e];
  if (threadIdx.x == 0) *status = (sweep >= max_sweeps) ? 1 : 0;
}

// Column norms (one block per column), descending ranks (ties by index) and the
// scattered outputs U[:, rank_j] = a_j / |a_j|, S[rank_j] = |a_j|, V[:, rank_j] = v_j.
__global__ void col_norms_kernel(const double* Ac, int64_t m, double* sig) {
  __shared__ double red[32];
  const int j = blockIdx.x;
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) { double x = Ac[int64_t(j) * m + i]; acc = fma(x, x, acc); }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) t += red[w];
    sig[j] = sqrt(t);
  }
}

__global__ void rank_kernel(const double* sig, int n, int* rank, double* S) {
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    int rk = 0;
    for (int i = 0; i < n; ++i) rk += (sig[i] > sig[j]) || (sig[i] == sig[j] && i < j);
    rank[j] = rk;
    S[rk] = sig[j];
  }
}

__global__ void svd_scatter_kernel(const double* Ac, int64_t m, int n, int N, const double* Vc,
                                   const double* sig, const int* rank, double* U, double* V) {
  const int64_t tu = m * n, tv = int64_t(n) * n;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < tu + tv;
       e += int64_t(gridDim.x) * blockDim.x) {
    if (e < tu) {
      int64_t i = e / n;
      int j = int(e - i * n);
      double sj = sig[j];
      U[i * n + rank[j]] = sj > 0.0 ? Ac[int64_t(j) * m + i] / sj : 0.0;
    } else {
      int64_t f = e - tu;
      int i = int(f / n), j = int(f % n);
      V[int64_t(i) * n + rank[j]] = Vc[int64_t(j) * N + i];
    }
  }
}

__global__ void to_colmajor_kernel(const double* A, int64_t m, int n, int N, double* Ac, double* Vc) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < m * N + int64_t(N) * N;
       e += int64_t(gridDim.x) * blockDim.x) {
    if (e < m * N) {
      int64_t j = e / m, i = e - (e / m) * m;
      Ac[e] = (j < n) ? A[i * n + j] : 0.0;
    } else {
      int64_t f = e - m * N;
      int64_t j = f / N, i = f - (f / N) * N;
      Vc[f] = (i == j) ? 1.0 : 0.0;
    }
  }
}

__global__ void transpose_kernel(const double* A, int64_t rows, int64_t cols, double* At) {
  __shared__ double tile[32][33];
  int64_t bx = int64_t(blockIdx.x) * 32, by = int64_t(blockIdx.y) * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    int64_t r = by + k, c = bx + threadIdx.x;
    if (r < rows && c < cols) tile[k][threadIdx.x] = A[r * cols + c];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    int64_t c = bx + k, r = by + threadIdx.x;
    if (r < rows && c < cols) At[c * rows + r] = tile[threadIdx.x][k];
  }
}

// Multi-block one-sided Jacobi for tall matrices: one launch per round of the
// round-robin schedule, one block per column pair, the block's threads split the rows.
__global__ void __launch_bounds__(256) tall_jacobi_round_kernel(double* Ac, int64_t m, int N,
                                                                double* Vc, int r, double tol,
                                                                const double* fro2, int* rotated) {
  __shared__ double red[3][8];
  __shared__ double cs[2];
  __shared__ int doit;
  const int k = blockIdx.x;
  int p, q;
  if (k == 0) { p = N - 1; q = r % (N - 1); }
  else { p = (r + k) % (N - 1); q = (r + N - 1 - k) % (N - 1); }
  double* ap = Ac + int64_t(p) * m;
  double* aq = Ac + int64_t(q) * m;
  double al = 0.0, be = 0.0, ga = 0.0;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
    double x = ap[i], y = aq[i];
    al = fma(x, x, al);
    be = fma(y, y, be);
    ga = fma(x, y, ga);
  }
  for (int o = 16; o > 0; o >>= 1) {
    al += __shfl_xor_sync(0xffffffffu, al, o);
    be += __shfl_xor_sync(0xffffffffu, be, o);
    ga += __shfl_xor_sync(0xffffffffu, ga, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { red[0][warp] = al; red[1][warp] = be; red[2][warp] = ga; }
  __syncthreads();
  if (threadIdx.x == 0) {
    al = be = ga = 0.0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) { al += red[0][w]; be += red[1][w]; ga += red[2][w]; }
    const double floor2 = 7.9e-31 * (*fro2);
    doit = (al > floor2 && be > floor2 && fabs(ga) > tol * sqrt(al) * sqrt(be)) ? 1 : 0;
    if (doit) {
      double zeta = (be - al) / (2.0 * ga);
      double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
      double c = 1.0 / sqrt(1.0 + t * t);
      cs[0] = c;
      cs[1] = c * t;
      *rotated = 1;
    }
  }
  __syncthreads();
  if (!doit) return;
  const double c = cs[0], sn = cs[1];
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
    double x = ap[i], y = aq[i];
    ap[i] = c * x - sn * y;
    aq[i] = sn * x + c * y;
  }
  double* vp = Vc + int64_t(p) * N;
  double* vq = Vc + int64_t(q) * N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    double x = vp[i], y = vq[i];
    vp[i] = c * x - sn * y;
    vq[i] = sn * x + c * y;
  }
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Time limit of one grid-barrier wait (2 s unless a caller changed it on this device).
__device__ unsigned long long g_barrier_limit_ns = 2000000000ull;

// Grid-wide barrier over co-resident blocks with a time limit.  bar[0] counts arrivals,
// bar[1] is the generation, bar[2] the abort flag.  Thread 0 of each block reads the
// generation, arrives, and the last block to arrive resets the count and advances the
// generation; the others wait for that, at most g_barrier_limit_ns, after which they set
// the abort flag.  Every block returns false once the abort flag is set, so no block
// waits for ever.
__device__ bool grid_barrier(unsigned* bar) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vb = bar;
    const unsigned gen = vb[1];
    __threadfence();
    if (atomicAdd(&bar[0], 1u) + 1u == gridDim.x) {
      atomicExch(&bar[0], 0u);
      __threadfence();
      atomicAdd(&bar[1], 1u);
      ok = 1;
    } else {
      const uint64_t t0 = global_ns(), limit = g_barrier_limit_ns;
      while (vb[1] == gen && vb[2] == 0u) {
        if (global_ns() - t0 >= limit) { atomicExch(&bar[2], 1u); break; }
        __nanosleep(64);
      }
      ok = vb[1] != gen;
    }
    __threadfence();
    if (vb[2] != 0u) ok = 0;
  }
  __syncthreads();
  return ok != 0;
}

constexpr int kCache = 4;  // column elements per thread kept in registers

// The same rotations as tall_jacobi_round_kernel, all sweeps in one cooperative launch:
// block b handles pairs b, b + gridDim.x, ... of each round and a grid-wide barrier
// separates rounds.  All blocks decide convergence from the same flag after a barrier.
// status: 0 converged, 1 not converged within max_sweeps, 2 a barrier timed out.
__global__ void __launch_bounds__(256) coop_jacobi_kernel(double* Ac, int64_t m, int N, double* Vc,
                                                          double tol, const double* fro2,
                                                          int* rotated, int* status,
                                                          int max_sweeps, unsigned* bar) {
  __shared__ double red[3][8];
  __shared__ double cs[2];
  __shared__ int doit;
  const double floor2 = 7.9e-31 * (*fro2);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int sweep = 0, converged = 0;
  for (; sweep < max_sweeps; ++sweep) {
    for (int r = 0; r < N - 1; ++r) {
      for (int k = blockIdx.x; k < N / 2; k += gridDim.x) {
        int p, q;
        if (k == 0) { p = N - 1; q = r % (N - 1); }
        else { p = (r + k) % (N - 1); q = (r + N - 1 - k) % (N - 1); }
        double* ap = Ac + int64_t(p) * m;
        double* aq = Ac + int64_t(q) * m;
        double* vp = Vc + int64_t(p) * N;
        double* vq = Vc + int64_t(q) * N;
        // short columns stay in registers from the inner products to the rotation, and the
        // V columns are fetched before the inner products so their latency overlaps them
        const bool cached = m <= kCache * int64_t(blockDim.x) && N <= kCache * int(blockDim.x);
        double xs[kCache], ys[kCache], vxs[kCache], vys[kCache];
        double al = 0.0, be = 0.0, ga = 0.0;
        if (cached) {
#pragma unroll
          for (int c = 0; c < kCache; ++c) {
            const int i = threadIdx.x + c * blockDim.x;
            vxs[c] = i < N ? vp[i] : 0.0;
            vys[c] = i < N ? vq[i] : 0.0;
          }
#pragma unroll
          for (int c = 0; c < kCache; ++c) {
            const int64_t i = threadIdx.x + int64_t(c) * blockDim.x;
            xs[c] = i < m ? ap[i] : 0.0;
            ys[c] = i < m ? aq[i] : 0.0;
          }
#pragma unroll
          for (int c = 0; c < kCache; ++c) {
            if (threadIdx.x + int64_t(c) * blockDim.x < m) {
              al = fma(xs[c], xs[c], al);
              be = fma(ys[c], ys[c], be);
              ga = fma(xs[c], ys[c], ga);
            }
          }
        } else {
          for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
            double x = ap[i], y = aq[i];
            al = fma(x, x, al);
            be = fma(y, y, be);
            ga = fma(x, y, ga);
          }
        }
        for (int o = 16; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        if (lane == 0) { red[0][warp] = al; red[1][warp] = be; red[2][warp] = ga; }
        __syncthreads();
        if (threadIdx.x == 0) {
          al = be = ga = 0.0;
          for (int w = 0; w < int(blockDim.x >> 5); ++w) { al += red[0][w]; be += red[1][w]; ga += red[2][w]; }
          doit = (al > floor2 && be > floor2 && fabs(ga) > tol * sqrt(al) * sqrt(be)) ? 1 : 0;
          if (doit) {
            double zeta = (be - al) / (2.0 * ga);
            double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            double c = 1.0 / sqrt(1.0 + t * t);
            cs[0] = c;
            cs[1] = c * t;
            atomicExch(rotated, 1);
          }
        }
        __syncthreads();
        if (doit) {
          const double c = cs[0], sn = cs[1];
          if (cached) {
#pragma unroll
            for (int cc = 0; cc < kCache; ++cc) {
              const int64_t i = threadIdx.x + int64_t(cc) * blockDim.x;
              if (i < m) {
                const double x = xs[cc], y = ys[cc];
                ap[i] = c * x - sn * y;
                aq[i] = sn * x + c * y;
              }
            }
#pragma unroll
            for (int cc = 0; cc < kCache; ++cc) {
              const int i = threadIdx.x + cc * blockDim.x;
              if (i < N) {
                const double x = vxs[cc], y = vys[cc];
                vp[i] = c * x - sn * y;
                vq[i] = sn * x + c * y;
              }
            }
          } else {
            for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
              double x = ap[i], y = aq[i];
              ap[i] = c * x - sn * y;
              aq[i] = sn * x + c * y;
            }
            for (int i = threadIdx.x; i < N; i += blockDim.x) {
              double x = vp[i], y = vq[i];
              vp[i] = c * x - sn * y;
              vq[i] = sn * x + c * y;
            }
          }
        }
        __syncthreads();
      }
      if (!grid_barrier(bar)) goto timed_out;
    }
    {
      const int any = atomicAdd(rotated, 0);
      if (!grid_barrier(bar)) goto timed_out;  // every block has read the flag
      if (blockIdx.x == 0 && threadIdx.x == 0) *rotated = 0;
      if (!grid_barrier(bar)) goto timed_out;
      if (!any) { converged = 1; break; }
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *status = converged ? 0 : 1;
  return;
timed_out:
  if (threadIdx.x == 0) atomicExch(status, 2);
}

__global__ void sumsq_kernel(const double* x, int64_t n, double* out) {
  double acc = 0.0;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n;
       e += int64_t(gridDim.x) * blockDim.x)
    acc = fma(x[e], x[e], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}
__device__ __forceinline__ double warp_sum(double x) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Householder QR with column pivoting, A P = Q R (Businger & Golub 1965), of a row-major
// m x n matrix (m >= n, m n <= kQrcpMaxElems), one block with the matrix in shared memory
// (column-major).  Step k takes the remaining column of largest norm (ties: lowest index),
// reflects rows k.. of it onto alpha e_k (alpha = -sign(x_0) ||x||) and updates the columns
// to its right, one warp per column, recomputing their norms over rows k + 1.. in the same
// pass.  Outputs: X = R^T (row-major n x n, lower triangular), the thin Q (row-major m x n,
// formed in place by accumulating the reflectors backwards) and perm (column j of A P is
// column perm[j] of A).
constexpr int kQrcpMaxN = 160;
constexpr int64_t kQrcpMaxElems = 25600;  // 200 KB of shared memory
__global__ void __launch_bounds__(1024) qrcp_kernel(const double* A, int m, int n, double* X, double* Q,
                                                    int* perm) {
  extern __shared__ double W[];  // W[j * m + i] = column j, row i
  __shared__ double nrm2[kQrcpMaxN], tau_s[kQrcpMaxN], diag_s[kQrcpMaxN];
  __shared__ int piv[kQrcpMaxN];
  __shared__ int pick;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int e = tid; e < m * n; e += blockDim.x) {
    const int i = e / n, j = e - (e / n) * n;
    W[j * m + i] = A[e];
  }
  for (int j = tid; j < n; j += blockDim.x) piv[j] = j;
  __syncthreads();
  for (int j = warp; j < n; j += nw) {
    double acc = 0.0;
    for (int i = lane; i < m; i += 32) acc = fma(W[j * m + i], W[j * m + i], acc);
    acc = warp_sum(acc);
    if (lane == 0) nrm2[j] = acc;
  }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (warp == 0) {
      double best = -1.0;
      int bj = k;
      for (int j = k + lane; j < n; j += 32)
        if (nrm2[j] > best) { best = nrm2[j]; bj = j; }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
        if (ob > best || (ob == best && oj < bj)) { best = ob; bj = oj; }
      }
      if (lane == 0) pick = bj;
    }
    __syncthreads();
    const int p = pick;
    if (p != k) {
      for (int i = tid; i < m; i += blockDim.x) {
        const double t = W[k * m + i];
        W[k * m + i] = W[p * m + i];
        W[p * m + i] = t;
      }
      if (tid == 0) {
        const double t = nrm2[k];
        nrm2[k] = nrm2[p];
        nrm2[p] = t;
        const int ti = piv[k];
        piv[k] = piv[p];
        piv[p] = ti;
      }
    }
    __syncthreads();
    if (warp == 0) {
      double acc = 0.0;
      for (int i = k + lane; i < m; i += 32) acc = fma(W[k * m + i], W[k * m + i], acc);
      acc = warp_sum(acc);
      if (lane == 0) {
        const double x0 = W[k * m + k], normx = sqrt(acc);
        const double alpha = x0 >= 0.0 ? -normx : normx;
        const double v0 = x0 - alpha;  // no cancellation: v0 and x0 have the same sign
        const double vtv = acc - x0 * x0 + v0 * v0;
        diag_s[k] = alpha;
        tau_s[k] = vtv > 0.0 ? 2.0 / vtv : 0.0;
        W[k * m + k] = v0;  // the reflector v = x - alpha e_0 stays in column k, rows k..
      }
    }
    __syncthreads();
    const double tau = tau_s[k];
    for (int j = k + 1 + warp; j < n; j += nw) {
      double d = 0.0;
      for (int i = k + lane; i < m; i += 32) d = fma(W[k * m + i], W[j * m + i], d);
      d = warp_sum(d) * tau;
      double acc = 0.0;
      for (int i = k + lane; i < m; i += 32) {
        const double x = fma(-d, W[k * m + i], W[j * m + i]);
        W[j * m + i] = x;
        if (i > k) acc = fma(x, x, acc);
      }
      acc = warp_sum(acc);
      if (lane == 0) nrm2[j] = acc;
    }
    __syncthreads();
  }
  // X = R^T: R's strict upper part is in W above the diagonal, its diagonal in diag_s
  for (int e = tid; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e - (e / n) * n;
    X[e] = i > j ? W[i * m + j] : (i == j ? diag_s[i] : 0.0);
  }
  for (int j = tid; j < n; j += blockDim.x) perm[j] = piv[j];
  __syncthreads();
  for (int e = tid; e < m * n; e += blockDim.x) {  // clear R: Q has zeros above the diagonal
    const int j = e / m, i = e - (e / m) * m;
    if (i < j) W[e] = 0.0;
  }
  __syncthreads();
  // Q = H_0 (H_1 (... (H_{n-1} [I; 0]))): at stage k the columns right of k hold the product of
  // the later reflectors (zero in rows <= k); apply H_k to them, then replace the reflector in
  // column k by H_k e_k
  for (int k = n - 1; k >= 0; --k) {
    const double tau = tau_s[k], v0 = W[k * m + k];
    for (int j = k + 1 + warp; j < n; j += nw) {
      double d = 0.0;
      for (int i = k + lane; i < m; i += 32) d = fma(W[k * m + i], W[j * m + i], d);
      d = warp_sum(d) * tau;
      for (int i = k + lane; i < m; i += 32) W[j * m + i] = fma(-d, W[k * m + i], W[j * m + i]);
    }
    __syncthreads();
    for (int i = k + tid; i < m; i += blockDim.x) W[k * m + i] = (i == k ? 1.0 : 0.0) - tau * v0 * W[k * m + i];
    __syncthreads();
  }
  for (int e = tid; e < m * n; e += blockDim.x) {
    const int i = e / n, j = e - (e / n) * n;
    Q[e] = W[j * m + i];
  }
}

// V[perm[j], :] = Ux[j, :] (n x n, row-major)
__global__ void permute_rows_kernel(const double* Ux, const int* perm, int n, double* V) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) {
    const int j = e / n, c = e - (e / n) * n;
    V[int64_t(perm[j]) * n + c] = Ux[e];
  }
}

// The single-block Jacobi keeps the whole m x N column-major copy in shared memory
// (at most 200 KB); it is used for narrow matrices (N < 32) that fit.  Everything else,
// including N = 2 with a tall m, takes the multi-block kernels, which handle one column
// pair as well.
bool single_block_fits(int64_t m, int N) { return N < 32 && m * N * int64_t(sizeof(double)) <= 200 * 1024; }
}  // namespace

int cholesky_max_n() { return kCholMaxN; }

void cholesky(const double* G, int n, double* R, int* status_dev, double shift_rel,
              cudaStream_t s) {
  check_extent(G, int64_t(n) * n - 1, sizeof(double), "cholesky input");
  check_extent(R, int64_t(n) * n - 1, sizeof(double), "cholesky output");
  TATRG_CHECK(n >= 1 && n <= kCholMaxN, TATRG_EINVAL, "cholesky: n must be <= 168");
  const size_t sm = size_t(n) * n * sizeof(double);
  ensure_smem_attr(reinterpret_cast<const void*>(cholesky_kernel), kCholMaxN * kCholMaxN * 8);
  cholesky_kernel<<<1, 1024, sm, s>>>(G, n, R, status_dev, shift_rel);
  TATRG_CUDA(cudaGetLastError());
}

void tri_inverse(const double* R, int n, double* Rinv, cudaStream_t s) {
  check_extent(R, int64_t(n) * n - 1, sizeof(double), "tri_inverse input");
  check_extent(Rinv, int64_t(n) * n - 1, sizeof(double), "tri_inverse output");
  TATRG_CHECK(n >= 1 && n <= 1024, TATRG_EINVAL, "tri_inverse: n must be <= 1024");
  if (n <= 160) {
    ensure_smem_attr(reinterpret_cast<const void*>(tri_inverse_kernel<true>), (160 * 160 + 4 * 160) * 8);
    tri_inverse_kernel<true><<<(n + 3) / 4, 128, size_t(n * n + 4 * n) * sizeof(double), s>>>(R, n, Rinv);
  } else {
    tri_inverse_kernel<false><<<(n + 3) / 4, 128, 4 * n * sizeof(double), s>>>(R, n, Rinv);
  }
  TATRG_CUDA(cudaGetLastError());
}

void jacobi_svd(const double* A, int64_t m, int n, double* U, double* S, double* V,
                int* status_dev, cudaStream_t s, Stats* st) {
  TATRG_CHECK(m >= n && n >= 1 && n <= 1024, TATRG_EINVAL, "jacobi_svd: need m >= n, 1 <= n <= 1024");
  check_extent(A, m * n - 1, sizeof(double), "jacobi input");
  check_extent(U, m * n - 1, sizeof(double), "jacobi U");
  check_extent(S, n - 1, sizeof(double), "jacobi S");
  check_extent(V, int64_t(n) * n - 1, sizeof(double), "jacobi V");
  const int N = n + (n & 1);
  DevBuf ac(size_t(m) * N * sizeof(double), s), vc(size_t(N) * N * sizeof(double), s);
  int64_t tot = m * N + int64_t(N) * N;
  to_colmajor_kernel<<<int(std::min<int64_t>(cdiv(tot, 256), 2048)), 256, 0, s>>>(A, m, n, N,
                                                                                  ac.d(), vc.d());
  TATRG_CUDA(cudaGetLastError());
  const double tol = std::max(1e-15, 2.220446049250313e-16 * std::sqrt(double(m)));
  if (single_block_fits(m, N)) {
    int threads = 32 * std::max(1, std::min(32, N / 2));
    ensure_smem_attr(reinterpret_cast<const void*>(jacobi_kernel), 200 * 1024);
    jacobi_kernel<<<1, threads, size_t(m * N) * sizeof(double), s>>>(ac.d(), m, N, vc.d(), 60, tol, status_dev);
    TATRG_CUDA(cudaGetLastError());
  } else {
    // one block per column pair, all sweeps in one cooperative launch (its blocks are
    // co-resident by construction; the barrier between rounds gives up after 2 s and
    // reports status 2)
    DevBuf aux(4 * sizeof(double), s);
    double* fro2 = aux.d();
    int* rot = reinterpret_cast<int*>(aux.d() + 1);
    unsigned* bar = reinterpret_cast<unsigned*>(aux.d() + 2);
    TATRG_CUDA(cudaMemsetAsync(aux.d(), 0, 4 * sizeof(double), s));
    sumsq_kernel<<<int(std::min<int64_t>(cdiv(m * N, 256), 1024)), 256, 0, s>>>(ac.d(), m * N, fro2);
    TATRG_CUDA(cudaGetLastError());
    int thr = m >= 256 ? 256 : (m >= 128 ? 128 : 64);
    int dev = 0, sms = 0, per_sm = 0;
    TATRG_CUDA(cudaGetDevice(&dev));
    TATRG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    TATRG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, coop_jacobi_kernel, thr, 0));
    const int blocks = std::max(1, std::min(N / 2, per_sm * sms));
    int max_sweeps = 60;
    double tol_ = tol;
    double* acp = ac.d();
    double* vcp = vc.d();
    int64_t m_ = m;
    int N_ = N;
    void* args[] = {&acp, &m_, &N_, &vcp, &tol_, &fro2, &rot, &status_dev, &max_sweeps, &bar};
    TATRG_CUDA(cudaLaunchCooperativeKernel((void*)coop_jacobi_kernel, dim3(blocks), dim3(thr), args, 0, s));
    if (st) st->launches += 1;
  }
  DevBuf sig(n * sizeof(double), s), rk(n * sizeof(int), s);
  col_norms_kernel<<<n, 256, 0, s>>>(ac.d(), m, sig.d());
  rank_kernel<<<1, 1024, 0, s>>>(sig.d(), n, rk.as<int>(), S);
  int64_t tot2 = m * n + int64_t(n) * n;
  svd_scatter_kernel<<<int(std::min<int64_t>(cdiv(tot2, 256), int64_t(sm_count()) * 16)), 256, 0, s>>>(
      ac.d(), m, n, N, vc.d(), sig.d(), rk.as<int>(), U, V);
  TATRG_CUDA(cudaGetLastError());
  if (st) st->launches += 5;
}

// ---------------------------------------------------------------------------------
// Jacobi SVD without device allocation.
//
// Its whole workspace (the column-major copy of A, the accumulated V, the column norms and
// ranks, the rotation and convergence flags) lives in one file-scope device array of
// kSvdScratchDoubles doubles (2 MiB), which every GPU that loads this library keeps until
// the process exits.  Host code may not hand the array's name to a kernel (on the host it
// is only a stand-in for the device symbol), so the device address is looked up once per
// device with cudaGetSymbolAddress, on the first call made with that device current.
// All calls share the array: concurrent calls whose work overlaps on the GPU race, and
// each call rewrites every part it reads before reading it.
namespace {
constexpr int64_t kSvdScratchDoubles = int64_t(1) << 18;
static __device__ __align__(256) double g_svd_scratch[kSvdScratchDoubles];

std::mutex g_svd_scratch_mu;
std::map<int, double*> g_svd_scratch_addr;  // device ordinal -> device address

double* svd_scratch_address() {
  int dev = 0;
  TATRG_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(g_svd_scratch_mu);
  auto it = g_svd_scratch_addr.find(dev);
  if (it != g_svd_scratch_addr.end()) return it->second;
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_svd_scratch);
  TATRG_CHECK(e == cudaSuccess && p != nullptr, TATRG_ECUDA,
              std::string("cudaGetSymbolAddress(svd scratch): ") + cudaGetErrorString(e));
  g_svd_scratch_addr[dev] = static_cast<double*>(p);
  return static_cast<double*>(p);
}
}  // namespace

int64_t svd_noalloc_scratch_needed(int64_t m, int n) {
  const int64_t N = n + (n & 1);
  // A copy, V, column norms, ranks (as doubles), ||A||_F^2, rotation flag, status
  return m * N + N * N + N + N + 3;
}

void jacobi_svd_noalloc(const double* A, int64_t m, int n, double* U, double* S, double* V,
                        cudaStream_t s) {
  TATRG_CHECK(m >= n && n >= 1 && n <= 1024, TATRG_EINVAL, "svd_noalloc: need m >= n, 1 <= n <= 1024");
  const int64_t need = svd_noalloc_scratch_needed(m, n);
  TATRG_CHECK(need <= kSvdScratchDoubles, TATRG_EINVAL,
              "svd_noalloc: m x n too large for the fixed scratch: needs (m + N + 2) * N + 3 <= "
              "262144 doubles, N = n rounded up to even");
  double* base = svd_scratch_address();
  const int N = n + (n & 1);
  double* ac = base;
  double* vc = ac + m * N;
  double* sig = vc + int64_t(N) * N;
  int* rk = reinterpret_cast<int*>(sig + N);
  double* fro2 = sig + 2 * N;
  int* rot = reinterpret_cast<int*>(fro2 + 1);
  int* status = reinterpret_cast<int*>(fro2 + 2);
  int64_t tot = m * N + int64_t(N) * N;
  to_colmajor_kernel<<<int(std::min<int64_t>(cdiv(tot, 256), 2048)), 256, 0, s>>>(A, m, n, N, ac, vc);
  TATRG_CUDA(cudaGetLastError());
  const double tol = std::max(1e-15, 2.220446049250313e-16 * std::sqrt(double(m)));
  int converged = 0;
  if (single_block_fits(m, N)) {
    int threads = 32 * std::max(1, std::min(32, N / 2));
    TATRG_CUDA(cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    jacobi_kernel<<<1, threads, size_t(m * N) * sizeof(double), s>>>(ac, m, N, vc, 60, tol, status);
    TATRG_CUDA(cudaGetLastError());
    int h = 1;
    TATRG_CUDA(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s));
    TATRG_CUDA(cudaStreamSynchronize(s));
    converged = (h == 0);
  } else {
    TATRG_CUDA(cudaMemsetAsync(fro2, 0, sizeof(double), s));
    sumsq_kernel<<<int(std::min<int64_t>(cdiv(m * N, 256), 1024)), 256, 0, s>>>(ac, m * N, fro2);
    TATRG_CUDA(cudaGetLastError());
    const int thr = m >= 256 ? 256 : (m >= 128 ? 128 : 64);
    for (int sweep = 0; sweep < 60 && !converged; ++sweep) {
      TATRG_CUDA(cudaMemsetAsync(rot, 0, sizeof(int), s));
      for (int r = 0; r < N - 1; ++r) {
        tall_jacobi_round_kernel<<<N / 2, thr, 0, s>>>(ac, m, N, vc, r, tol, fro2, rot);
        TATRG_CUDA(cudaGetLastError());
      }
      int h = 0;
      TATRG_CUDA(cudaMemcpyAsync(&h, rot, sizeof(int), cudaMemcpyDeviceToHost, s));
      TATRG_CUDA(cudaStreamSynchronize(s));
      converged = (h == 0);
    }
  }
  TATRG_CHECK(converged, TATRG_ENUMERIC, "svd_noalloc: Jacobi SVD did not converge");
  col_norms_kernel<<<n, 256, 0, s>>>(ac, m, sig);
  rank_kernel<<<1, 1024, 0, s>>>(sig, n, rk, S);
  int64_t tot2 = m * n + int64_t(n) * n;
  svd_scatter_kernel<<<int(std::min<int64_t>(cdiv(tot2, 256), int64_t(sm_count()) * 16)), 256, 0, s>>>(ac, m, n, N, vc,
                                                                                       sig, rk, U, V);
  TATRG_CUDA(cudaGetLastError());
  TATRG_CUDA(cudaStreamSynchronize(s));
}

// SVD of a square A through a pivoted QR of its transpose (Drmac & Veselic, SIAM J. Matrix
// Anal. Appl. 29, 2008): A^T P = Q R, then one-sided Jacobi on X = R^T, X = Ux S Vx^T, so
// A = P X Q^T = (P Ux) S (Q Vx)^T.  Pivoting puts the large columns first and the rows of R
// are graded, so the Jacobi sweeps on R^T converge in a few sweeps where the Jacobi on A
// takes tens.  Factoring A^T keeps the conventions of jacobi_svd: V is a full orthonormal
// basis and the columns of U that belong to zero singular values are zero.
bool qrcp_svd_fits(int64_t m, int n) {
  // measured on the chi = 48 step, the pivoted QR (one block) costs more than the Jacobi
  // sweeps it saves on the step's spectra, so it is used only when TATRG_SVD_QRCP=1
  static const bool on = []() {
    const char* e = getenv("TATRG_SVD_QRCP");
    return e && e[0] == '1';
  }();
  return on && n >= 32 && n <= kQrcpMaxN && m == n;
}

void jacobi_svd_qrcp(const double* A, int64_t m, int n, double* U, double* S, double* V, int* status_dev,
                     cudaStream_t s, Stats* st) {
  TATRG_CHECK(qrcp_svd_fits(m, n), TATRG_EINVAL, "jacobi_svd_qrcp: size out of range");
  check_extent(A, m * n - 1, sizeof(double), "qrcp input");
  check_extent(U, m * n - 1, sizeof(double), "qrcp U");
  check_extent(V, int64_t(n) * n - 1, sizeof(double), "qrcp V");
  DevBuf At(size_t(n) * n * sizeof(double), s), X(size_t(n) * n * sizeof(double), s),
      Qm(size_t(n) * n * sizeof(double), s), perm(size_t(n) * sizeof(int), s),
      Ux(size_t(n) * n * sizeof(double), s), Vx(size_t(n) * n * sizeof(double), s);
  transpose(A, n, n, At.d(), s);
  ensure_smem_attr(reinterpret_cast<const void*>(qrcp_kernel), int(kQrcpMaxElems * sizeof(double)));
  qrcp_kernel<<<1, 1024, size_t(n) * n * sizeof(double), s>>>(At.d(), n, n, X.d(), Qm.d(), perm.as<int>());
  TATRG_CUDA(cudaGetLastError());
  jacobi_svd(X.d(), n, n, Ux.d(), S, Vx.d(), status_dev, s, st);
  GemmDesc g;  // V = Q Vx
  g.m = modes({{n, n, n}});
  g.n = modes({{n, 1, 1}});
  g.k = modes({{n, 1, n}});
  gemm_f64(g, Qm.d(), Vx.d(), V, s, st);
  permute_rows_kernel<<<int(std::max<int64_t>(1, std::min<int64_t>(cdiv(int64_t(n) * n, 256), 64))), 256, 0, s>>>(
      Ux.d(), perm.as<int>(), n, U);  // U[perm[j], :] = Ux[j, :]
  TATRG_CUDA(cudaGetLastError());
  if (st) st->launches += 2;
}

void set_barrier_limit_ns(unsigned long long ns) {
  TATRG_CUDA(cudaMemcpyToSymbol(g_barrier_limit_ns, &ns, sizeof(ns)));
}

void transpose(const double* A, int64_t rows, int64_t cols, double* At, cudaStream_t s) {
  if (rows == 0 || cols == 0) return;
  check_extent(A, rows * cols - 1, sizeof(double), "transpose input");
  check_extent(At, rows * cols - 1, sizeof(double), "transpose output");
  dim3 grid(unsigned(cdiv(cols, 32)), unsigned(cdiv(rows, 32)));
  transpose_kernel<<<grid, dim3(32, 8), 0, s>>>(A, rows, cols, At);
  TATRG_CUDA(cudaGetLastError());
}

}  // namespace tatrg
