// Device-side D2Q9 lattice constants and the pseudopotential psi(rho).
#pragma once
#include <cuda_runtime.h>

#include "lbm_internal.h"

namespace lbm {

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

// psi(rho): exponential psi0 exp(-rho0/rho) (Sec. 3.2) or the Carnahan-Starling form
// sqrt(2 (p - rho/3)/G); zero for a single-phase fluid.
template <typename C, int EOS>
__device__ __forceinline__ C psi_of(const Consts<C>& k, C rho) {
  if constexpr (EOS == LBM_EOS_EXP) {
    return k.psi0 * exp(-k.rho0 / rho);
  } else if constexpr (EOS == LBM_EOS_CS) {
    const C eta = k.b4 * rho;
    const C om = C(1) - eta;
    const C num = C(1) + eta + eta * eta - eta * eta * eta;
    const C pr = rho * k.RT * num / (om * om * om) - k.a * rho * rho;
    return sqrt((pr - rho * C(1.0 / 3.0)) * k.two_over_G);
  } else {
    return C(0);
  }
}

}  // namespace lbm
