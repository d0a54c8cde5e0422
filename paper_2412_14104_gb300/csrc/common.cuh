// Shared declarations of the tatrg CUDA library: status plumbing, device buffers and the
// multi-mode contraction descriptor that every GEMM back-end consumes.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <map>
#include <mutex>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/tatrg.h"

namespace tatrg {

// Exception carried up to the C-ABI boundary, where it becomes a tatrg_status.
struct Error : public std::runtime_error {
  tatrg_status code;
  Error(tatrg_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define TATRG_CUDA(call)                                                              \
  do {                                                                                \
    cudaError_t e__ = (call);                                                         \
    if (e__ != cudaSuccess)                                                           \
      throw ::tatrg::Error(TATRG_ECUDA, std::string(#call) + ": " +                   \
                                            cudaGetErrorString(e__) + " at " +        \
                                            __FILE__ + ":" + std::to_string(__LINE__)); \
  } while (0)

#define TATRG_CHECK(cond, code, msg)                 \
  do {                                               \
    if (!(cond)) throw ::tatrg::Error((code), (msg)); \
  } while (0)

// Registry of the library's live device allocations.  Every launch that addresses a
// buffer through mode strides checks, on the host and before the launch, that the
// largest offset it can reach stays inside the allocation the base pointer belongs to.
struct AllocRegistry {
  std::mutex mu;
  std::map<uintptr_t, size_t> live;  // base -> bytes
  static AllocRegistry& get() {
    static AllocRegistry r;
    return r;
  }
  void add(void* p, size_t n) {
    std::lock_guard<std::mutex> l(mu);
    live[reinterpret_cast<uintptr_t>(p)] = n;
  }
  void remove(void* p) {
    std::lock_guard<std::mutex> l(mu);
    live.erase(reinterpret_cast<uintptr_t>(p));
  }
  // true when [p, p + bytes) lies inside one registered allocation, or p is not ours
  bool inside(const void* p, size_t bytes) {
    std::lock_guard<std::mutex> l(mu);
    uintptr_t a = reinterpret_cast<uintptr_t>(p);
    auto it = live.upper_bound(a);
    if (it == live.begin()) return true;  // foreign pointer (caller-owned)
    --it;
    if (a >= it->first + it->second) return true;  // foreign pointer
    return a + bytes <= it->first + it->second;
  }
};

inline void check_extent(const void* p, int64_t max_elem, size_t esize, const char* what) {
  if (!AllocRegistry::get().inside(p, size_t(max_elem + 1) * esize))
    throw Error(TATRG_EINVAL, std::string("out-of-range operand extent in ") + what);
}

// Stream-ordered device buffer (cudaMallocAsync pool); frees on the same stream.
class DevBuf {
 public:
  DevBuf() = default;
  DevBuf(size_t bytes, cudaStream_t s) { alloc(bytes, s); }
  ~DevBuf() { release(); }
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p_(o.p_), n_(o.n_), s_(o.s_) { o.p_ = nullptr; o.n_ = 0; }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) { release(); p_ = o.p_; n_ = o.n_; s_ = o.s_; o.p_ = nullptr; o.n_ = 0; }
    return *this;
  }
  void alloc(size_t bytes, cudaStream_t s) {
    release();
    s_ = s;
    n_ = bytes;
    if (bytes) {
      cudaError_t e = cudaMallocAsync(&p_, bytes, s);
      if (e != cudaSuccess) {
        p_ = nullptr;
        cudaGetLastError();  // an allocation failure is not sticky: clear it for later checks
        throw Error(TATRG_ENOMEM, "cudaMallocAsync(" + std::to_string(bytes) + "): " +
                                      cudaGetErrorString(e));
      }
      AllocRegistry::get().add(p_, bytes);
    }
  }
  void release() {
    if (p_) {
      AllocRegistry::get().remove(p_);
      cudaFreeAsync(p_, s_);
    }
    p_ = nullptr;
    n_ = 0;
  }
  // Free on stream s instead of the allocating stream (s must be ordered after every use).
  void rebind(cudaStream_t s) { s_ = s; }
  template <class T> T* as() const { return reinterpret_cast<T*>(p_); }
  double* d() const { return reinterpret_cast<double*>(p_); }
  size_t bytes() const { return n_; }
  bool empty() const { return p_ == nullptr; }

 private:
  void* p_ = nullptr;
  size_t n_ = 0;
  cudaStream_t s_ = 0;
};

inline DevBuf dalloc(int64_t n_doubles, cudaStream_t s) {
  return DevBuf(size_t(n_doubles > 0 ? n_doubles : 1) * sizeof(double), s);
}

// ---------------------------------------------------------------------------------
// A multi-mode index: a flat index 0..prod(ext)-1 decomposed outermost-first into up to
// kMaxModes sub-indices, each carrying its own element stride in the operands.
constexpr int kMaxModes = 4;

struct ModeIdx {
  int n = 0;                       // number of modes (0 means a single index of extent 1)
  int64_t ext[kMaxModes] = {1, 1, 1, 1};
  int64_t s0[kMaxModes] = {0, 0, 0, 0};  // stride in the first operand that carries it
  int64_t s1[kMaxModes] = {0, 0, 0, 0};  // stride in the second operand that carries it
  int64_t total() const {
    int64_t t = 1;
    for (int i = 0; i < n; ++i) t *= ext[i];
    return t;
  }
};

// C[m, n] = alpha * sum_k A[m, k] B[k, n] + beta * C[m, n] with
//   M modes: (ext, strideA, strideC), N modes: (ext, strideB, strideC),
//   K modes: (ext, strideA, strideB).  All strides are in elements.
struct GemmDesc {
  ModeIdx m, n, k;
  double alpha = 1.0, beta = 0.0;
};

inline int64_t max_off0(const ModeIdx& x) {
  int64_t o = 0;
  for (int i = 0; i < x.n; ++i) o += (x.ext[i] - 1) * x.s0[i];
  return o;
}
inline int64_t max_off1(const ModeIdx& x) {
  int64_t o = 0;
  for (int i = 0; i < x.n; ++i) o += (x.ext[i] - 1) * x.s1[i];
  return o;
}

// Host check of a contraction's reach into A, B and C (elements of esize bytes).
inline void check_gemm(const GemmDesc& d, const void* A, const void* B, const void* C) {
  if (d.m.total() == 0 || d.n.total() == 0) return;
  check_extent(A, max_off0(d.m) + max_off0(d.k), sizeof(double), "operand A");
  check_extent(B, max_off0(d.n) + max_off1(d.k), sizeof(double), "operand B");
  check_extent(C, max_off1(d.m) + max_off1(d.n), sizeof(double), "result C");
}

// Builders -------------------------------------------------------------------------
struct Mode3 {
  int64_t ext, s0, s1;
};

inline ModeIdx modes(std::initializer_list<Mode3> l) {
  ModeIdx r;
  for (const auto& x : l) {
    if (x.ext == 1) continue;  // drop unit modes
    if (r.n == kMaxModes) throw Error(TATRG_EINVAL, "too many modes in a contraction");
    r.ext[r.n] = x.ext;
    r.s0[r.n] = x.s0;
    r.s1[r.n] = x.s1;
    r.n++;
  }
  // merge adjacent modes that are contiguous in both operands
  ModeIdx o;
  for (int i = 0; i < r.n; ++i) {
    if (o.n > 0 && o.s0[o.n - 1] == r.s0[i] * r.ext[i] && o.s1[o.n - 1] == r.s1[i] * r.ext[i]) {
      o.ext[o.n - 1] *= r.ext[i];
      o.s0[o.n - 1] = r.s0[i];
      o.s1[o.n - 1] = r.s1[i];
    } else {
      o.ext[o.n] = r.ext[i];
      o.s0[o.n] = r.s0[i];
      o.s1[o.n] = r.s1[i];
      o.n++;
    }
  }
  return o;
}

inline ModeIdx modes(const std::vector<Mode3>& v) {
  ModeIdx r;
  for (const auto& x : v) {
    if (x.ext == 1) continue;
    if (r.n == kMaxModes) throw Error(TATRG_EINVAL, "too many modes in a contraction");
    r.ext[r.n] = x.ext;
    r.s0[r.n] = x.s0;
    r.s1[r.n] = x.s1;
    r.n++;
  }
  ModeIdx o;  // merge adjacent modes that are contiguous in both operands
  for (int i = 0; i < r.n; ++i) {
    if (o.n > 0 && o.s0[o.n - 1] == r.s0[i] * r.ext[i] && o.s1[o.n - 1] == r.s1[i] * r.ext[i]) {
      o.ext[o.n - 1] *= r.ext[i];
      o.s0[o.n - 1] = r.s0[i];
      o.s1[o.n - 1] = r.s1[i];
    } else {
      o.ext[o.n] = r.ext[i];
      o.s0[o.n] = r.s0[i];
      o.s1[o.n] = r.s1[i];
      o.n++;
    }
  }
  return o;
}

// Device-side decomposition of a flat index into the two operand offsets.
struct DevModes {
  int n;
  int64_t ext[kMaxModes];
  int64_t s0[kMaxModes];
  int64_t s1[kMaxModes];
};

inline DevModes dev(const ModeIdx& x) {
  DevModes d;
  d.n = x.n;
  for (int i = 0; i < kMaxModes; ++i) {
    d.ext[i] = x.ext[i];
    d.s0[i] = x.s0[i];
    d.s1[i] = x.s1[i];
  }
  return d;
}

__host__ __device__ inline void mode_offsets(const DevModes& d, int64_t flat, int64_t& o0,
                                             int64_t& o1) {
  o0 = 0;
  o1 = 0;
#pragma unroll
  for (int j = 0; j < kMaxModes; ++j) {  // innermost mode first; static indices (no local copy)
    const int i = kMaxModes - 1 - j;
    if (i < d.n) {
      const int64_t e = d.ext[i];
      const int64_t q = flat / e;
      const int64_t r = flat - q * e;
      o0 += r * d.s0[i];
      o1 += r * d.s1[i];
      flat = q;
    }
  }
}

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace tatrg
