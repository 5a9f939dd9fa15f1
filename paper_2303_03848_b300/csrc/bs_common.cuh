// bs_common.cuh -- device-side data structures shared by the kernels of the
// Parareal/PINN library (sm_103a).
//
// Partitioned tridiagonal layout (used by the Crank-Nicolson fine propagator
// and the implicit Euler coarse propagator, Section 3.2 of the paper):
//   A CTA of T = NW*32 threads owns one grid.  The Nx-2 interior unknowns plus
//   one row for the Smax Dirichlet node are laid out on R = T*M rows, with
//   Np = R - (Nx-1) identity padding rows in front.  Thread t owns rows
//   t*M .. t*M+M-1: M-1 "inner" rows and the "interface" row t*M+M-1.  The
//   interface row of thread T-1 is the Dirichlet node at Smax.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace bsp {

constexpr int kPcrLevels = 5;  // PCR inside one warp: strides 1, 2, 4, 8, 16
constexpr int kMaxNW = 4;      // warps per grid
constexpr unsigned kFull = 0xffffffffu;

// One pricing instance as the kernels see it.
struct Inst {
  double K, sigma, r, T, Smax, dS;
  int32_t Nx, P, Mf, Mg;
  int32_t NW, M, R, Np;        // partition of the tridiagonal rows
  int64_t coef_cn, coef_ie;    // offsets (doubles) of the two coefficient blocks in the pool
  int64_t exp_cn, exp_ie;      // offsets of exp(-r m dtau) tables (Mf+1 / Mg+1 entries)
  int64_t state_off;           // offset of the instance in (P+1)*Nx arrays
  int64_t slice_off;           // offset of the instance in P*Nx arrays
  int64_t task_off;            // offset of the instance in per-slice arrays (P entries)
  int64_t task1_off;           // offset of the instance in per-boundary arrays (P+1 entries)
};

// Coefficient block of one (instance, propagator): all doubles.
//   rows  [q][k][t], q: 0 lambda, 1 mu, 2 sigma, 3 alpha, 4 beta, 5 1/sigma
//   iface [q][t],    q: 0 kappa, 1 nu, 2 sigma_p, 3 1/sigma_p, 4 A, 5 C
//   pcr   [q][t],    q: 0..4 m1 per level, 5..9 m2 per level, 10 1/diag
//   resp  [q][t],    q: 0 response to Y_{w-1}, 1 response to Y_w
//   G     [NW][NW]   inverse of the cross-warp interface system
__host__ __device__ inline int64_t coef_rows_off(int q, int k, int t, int M, int T) {
  return ((int64_t)q * M + k) * T + t;
}
__host__ __device__ inline int64_t coef_if_off(int q, int t, int M, int T) { return 6LL * M * T + (int64_t)q * T + t; }
__host__ __device__ inline int64_t coef_pcr_off(int q, int t, int M, int T) {
  return 6LL * M * T + 6LL * T + (int64_t)q * T + t;
}
__host__ __device__ inline int64_t coef_resp_off(int q, int t, int M, int T) {
  return 6LL * M * T + 17LL * T + (int64_t)q * T + t;
}
__host__ __device__ inline int64_t coef_G_off(int v, int u, int M, int T, int NW) {
  return 6LL * M * T + 19LL * T + (int64_t)v * NW + u;
}
__host__ __device__ inline int64_t coef_block_size(int M, int T, int NW) {
  return 6LL * M * T + 19LL * T + (int64_t)NW * NW;
}

// Per-instance Parareal control word, updated on the device.
struct Ctrl {
  int32_t done;        // 1 once converged / diverged / exhausted
  int32_t iterations;  // Parareal iterations done
  int32_t status;      // bs_status of the instance
  int32_t pad;
  double last_norm;
};

}  // namespace bsp
