// Device-side D2Q9 lattice constants and the pseudopotential psi(rho).
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "lbm_internal.h"

namespace lbm {

// Index checks of the debug build (-DLBM_CHECKED, the library variant liblbm_gb300_checked.so):
// an index outside [0, limit) is reported by device printf ("LBM_OOB <file>:<line> ...") and
// replaced by 0, so the access stays inside the buffer and the run continues.  In the normal
// build LBM_CHK(i, limit) is i.
#ifdef LBM_CHECKED
__device__ __noinline__ inline long long oob_report(long long i, long long limit,
                                                    const char* file, int line) {
  printf("LBM_OOB %s:%d index %lld limit %lld\n", file, line, i, limit);
  return 0;
}
#define LBM_CHK(i, limit)                                                             \
  ((long long)(i) >= 0 && (long long)(i) < (long long)(limit)                          \
       ? (i)                                                                            \
       : static_cast<decltype(i)>(oob_report((long long)(i), (long long)(limit), __FILE__, \
                                             __LINE__)))
#else
#define LBM_CHK(i, limit) (i)
#endif

// Directions 0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1) 5:(1,1) 6:(-1,1) 7:(-1,-1) 8:(1,-1).
__host__ __device__ constexpr int ex(int a) {
  return a == 1 || a == 5 || a == 8 ? 1 : (a == 3 || a == 6 || a == 7 ? -1 : 0);
}
__host__ __device__ constexpr int ey(int a) {
  return a == 2 || a == 5 || a == 6 ? 1 : (a == 4 || a == 7 || a == 8 ? -1 : 0);
}
// Opposite direction.
__host__ __device__ constexpr int opposite(int a) {
  return a == 1 ? 3 : a == 2 ? 4 : a == 3 ? 1 : a == 4 ? 2 : a == 5 ? 7 : a == 6 ? 8 : a == 7 ? 5 : a == 8 ? 6 : 0;
}
// Weights of Eq. (4): 4/9, 1/9 (axis), 1/36 (diagonal).
template <typename T>
__host__ __device__ constexpr T wgt(int a) {
  return a == 0 ? T(4.0 / 9.0) : (a <= 4 ? T(1.0 / 9.0) : T(1.0 / 36.0));
}
// Interaction weights of Eq. (16): 1/3 for |e|^2 = 1, 1/12 for |e|^2 = 2.
template <typename T>
__host__ __device__ constexpr T wpsi(int a) {
  return a == 0 ? T(0) : (a <= 4 ? T(1.0 / 3.0) : T(1.0 / 12.0));
}

__device__ __forceinline__ int wrap_once(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }
__device__ __forceinline__ int wrap_any(int v, int n) {
  int r = v % n;
  return r < 0 ? r + n : r;
}

// Storage of the nine populations of a lattice.  Element (a, n) of plane a at node n:
//   double  FP64 values, planes [a][n]
//   float   FP32 deviations f_a - w_a rho_ref, planes [a][n]
//   __half  mixed: plane 0 (the rest population, which never streams) as FP32 deviations, then
//           planes 1..8 as FP16 deviations; the rest population absorbs the rounding of the
//           moving ones, so mass stays at FP32 accuracy
template <typename S>
struct Pop;
template <>
struct Pop<double> {
  using C = double;
  static constexpr bool dev = false;
  static __device__ __forceinline__ C load(const void* b, int a, int N, int n) {
    return static_cast<const double*>(b)[a * N + LBM_CHK(n, N)];
  }
  static __device__ __forceinline__ C rounded(int a, C v) { return v; }
  static __device__ __forceinline__ void store(void* b, int a, int N, int n, C v) {
    static_cast<double*>(b)[a * N + LBM_CHK(n, N)] = v;
  }
  // element e = a N + n, in the arithmetic type C; store_t returns the value as stored
  static __device__ __forceinline__ C load_t(const void* b, int e, int N) {
    return static_cast<const double*>(b)[LBM_CHK(e, 9 * N)];
  }
  static __device__ __forceinline__ C store_t(void* b, int e, int N, C v) {
    static_cast<double*>(b)[LBM_CHK(e, 9 * N)] = v;
    return v;
  }
  static __device__ __forceinline__ double load_e(const void* b, int e, int N) {
    return static_cast<const double*>(b)[LBM_CHK(e, 9 * N)];
  }
  static __device__ __forceinline__ double store_e(void* b, int e, int N, double v) {
    static_cast<double*>(b)[LBM_CHK(e, 9 * N)] = v;
    return v;
  }
};
template <>
struct Pop<float> {
  using C = float;
  static constexpr bool dev = true;
  static __device__ __forceinline__ C load(const void* b, int a, int N, int n) {
    return static_cast<const float*>(b)[a * N + LBM_CHK(n, N)];
  }
  static __device__ __forceinline__ C rounded(int a, C v) { return v; }
  static __device__ __forceinline__ void store(void* b, int a, int N, int n, C v) {
    static_cast<float*>(b)[a * N + LBM_CHK(n, N)] = v;
  }
  static __device__ __forceinline__ C load_t(const void* b, int e, int N) {
    return static_cast<const float*>(b)[LBM_CHK(e, 9 * N)];
  }
  static __device__ __forceinline__ C store_t(void* b, int e, int N, C v) {
    static_cast<float*>(b)[LBM_CHK(e, 9 * N)] = v;
    return v;
  }
  static __device__ __forceinline__ double load_e(const void* b, int e, int N) {
    return double(static_cast<const float*>(b)[LBM_CHK(e, 9 * N)]);
  }
  static __device__ __forceinline__ double store_e(void* b, int e, int N, double v) {
    const float s = float(v);
    static_cast<float*>(b)[LBM_CHK(e, 9 * N)] = s;
    return double(s);
  }
};
template <>
struct Pop<__half> {
  using C = float;
  static constexpr bool dev = true;
  static __device__ __forceinline__ const __half* moving(const void* b, int N) {
    return reinterpret_cast<const __half*>(static_cast<const float*>(b) + N);
  }
  static __device__ __forceinline__ __half* moving(void* b, int N) {
    return reinterpret_cast<__half*>(static_cast<float*>(b) + N);
  }
  static __device__ __forceinline__ C load(const void* b, int a, int N, int n) {
    n = LBM_CHK(n, N);
    return a == 0 ? static_cast<const float*>(b)[n] : __half2float(moving(b, N)[(a - 1) * N + n]);
  }
  static __device__ __forceinline__ C rounded(int a, C v) {
    return a == 0 ? v : __half2float(__float2half_rn(v));
  }
  static __device__ __forceinline__ void store(void* b, int a, int N, int n, C v) {
    n = LBM_CHK(n, N);
    if (a == 0)
      static_cast<float*>(b)[n] = v;
    else
      moving(b, N)[(a - 1) * N + n] = __float2half_rn(v);
  }
  static __device__ __forceinline__ C load_t(const void* b, int e, int N) {
    e = LBM_CHK(e, 9 * N);
    return e < N ? static_cast<const float*>(b)[e] : __half2float(moving(b, N)[e - N]);
  }
  static __device__ __forceinline__ C store_t(void* b, int e, int N, C v) {
    e = LBM_CHK(e, 9 * N);
    if (e < N) {
      static_cast<float*>(b)[e] = v;
      return v;
    }
    const __half h = __float2half_rn(v);
    moving(b, N)[e - N] = h;
    return __half2float(h);
  }
  static __device__ __forceinline__ double load_e(const void* b, int e, int N) {
    e = LBM_CHK(e, 9 * N);
    return e < N ? double(static_cast<const float*>(b)[e])
                 : double(__half2float(moving(b, N)[e - N]));
  }
  static __device__ __forceinline__ double store_e(void* b, int e, int N, double v) {
    e = LBM_CHK(e, 9 * N);
    if (e < N) {
      const float s = float(v);
      static_cast<float*>(b)[e] = s;
      return double(s);
    }
    const __half h = __double2half(v);
    moving(b, N)[e - N] = h;
    return double(__half2float(h));
  }
};

// Lane types of the per-node arithmetic: one node (float, double) or two nodes packed in the
// f32x2 registers of Blackwell's paired FP32 instructions (float2).  Elem<L>::C is the element
// type; splat() broadcasts a scalar.
template <typename L>
struct Elem;
template <>
struct Elem<float> { using C = float; static constexpr int W = 1; };
template <>
struct Elem<double> { using C = double; static constexpr int W = 1; };
template <>
struct Elem<float2> { using C = float; static constexpr int W = 2; };
template <typename L>
__device__ __forceinline__ L splat(typename Elem<L>::C c) {
  if constexpr (Elem<L>::W == 2) return make_float2(c, c); else return c;
}

// psi(rho): exponential psi0 exp(-rho0/rho) (Sec. 3.2) or the Carnahan-Starling form
// sqrt(2 (p - rho/3)/G); zero for a single-phase fluid.
// Division, reciprocal, square root and exponential in the arithmetic type: correctly rounded
// in FP64; in FP32 the hardware approximations (relative error of a few 2^-24, well inside the
// FP32 error budget of the method's steady state) to keep the FP32 step memory-bound.
__device__ __forceinline__ double q_div(double a, double b) { return a / b; }
__device__ __forceinline__ float q_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ float2 q_div(float2 a, float2 b) {
  return make_float2(__fdividef(a.x, b.x), __fdividef(a.y, b.y));
}
__device__ __forceinline__ double q_rcp(double a) { return 1.0 / a; }
__device__ __forceinline__ float q_rcp(float a) { return __fdividef(1.0f, a); }
__device__ __forceinline__ float2 q_rcp(float2 a) { return make_float2(q_rcp(a.x), q_rcp(a.y)); }
__device__ __forceinline__ double q_sqrt(double a) { return sqrt(a); }
__device__ __forceinline__ float q_sqrt(float a) { return a > 0.f ? __fmul_rn(a, rsqrtf(a)) : 0.f; }
__device__ __forceinline__ float2 q_sqrt(float2 a) { return make_float2(q_sqrt(a.x), q_sqrt(a.y)); }
__device__ __forceinline__ double q_exp(double a) { return exp(a); }
__device__ __forceinline__ float q_exp(float a) { return __expf(a); }
__device__ __forceinline__ float2 q_exp(float2 a) { return make_float2(__expf(a.x), __expf(a.y)); }

// Explicitly rounded arithmetic (no contraction freedom for the compiler): every kernel that
// inlines the per-node arithmetic (the scalar and the vectorised tile cores, the batched kernel)
// then produces the same bits for the same node.  The paired FP32 forms round each element
// exactly as the scalar ones; a - b is fma(b, -1, a), the same single rounding of a - b.
__device__ __forceinline__ float r_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double r_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float2 r_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float r_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double r_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float2 r_sub(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
__device__ __forceinline__ float r_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double r_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float2 r_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float r_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double r_fma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float2 r_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

template <typename C, int EOS, typename L>
__device__ __forceinline__ L psi_of(const Consts<C>& k, L rho) {
  if constexpr (EOS == LBM_EOS_EXP) {
    return r_mul(splat<L>(k.psi0), q_exp(r_mul(splat<L>(C(-1)), q_div(splat<L>(k.rho0), rho))));
  } else if constexpr (EOS == LBM_EOS_CS) {
    // p = rho R T (1 + eta + eta^2 - eta^3) / (1 - eta)^3 - a rho^2,  eta = b rho / 4, so
    // p - rho/3 = rho [R T num / (1 - eta)^3 - a rho - 1/3] with the numerator in Horner form
    // num = 1 + eta (1 + eta (1 - eta))
    const L one = splat<L>(C(1));
    const L eta = r_mul(splat<L>(k.b4), rho);
    const L om = r_sub(one, eta);
    const L num = r_fma(eta, r_fma(eta, om, one), one);
    const L om3 = r_mul(r_mul(om, om), om);
    const L inner = r_fma(splat<L>(k.RT), q_div(num, om3),
                          r_fma(splat<L>(-k.a), rho, splat<L>(C(-1.0 / 3.0))));
    return q_sqrt(r_mul(r_mul(rho, splat<L>(k.two_over_G)), inner));
  } else {
    return splat<L>(C(0));
  }
}

}  // namespace lbm
