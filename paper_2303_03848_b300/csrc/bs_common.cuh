// bs_common.cuh -- device-side data structures shared by the kernels of the
// Parareal/PINN library (sm_103a).
//
// Partitioned tridiagonal layout (used by the Crank-Nicolson fine propagator
// and the implicit Euler coarse propagator, Section 3.2 of the paper):
//   One grid (one time slice of one instance) is owned by a cluster of C CTAs
//   of NW warps each: GT = C*NW*32 threads, Ws = C*NW warps.  The Nx-2 interior
//   unknowns plus one row for the Smax Dirichlet node are laid out on
//   R = GT*M rows with Np = R - (Nx-1) identity padding rows in front.  Global
//   thread g (= cluster rank * NW*32 + threadIdx.x) owns rows g*M .. g*M+M-1:
//   M-1 "inner" rows and the "interface" row g*M+M-1.  Lane 31 of every warp
//   carries the warp-level interface unknown Y_w; the interface row of the last
//   thread of the cluster is the Dirichlet node at Smax.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace bsp {

constexpr int kPcrLevels = 5;  // PCR inside one warp: strides 1, 2, 4, 8, 16
constexpr int kMaxWs = 64;     // warps per grid (cluster of up to 16 CTAs x 4 warps)
constexpr unsigned kFull = 0xffffffffu;

// Bring the line holding p (global memory) into L2; a hint, with no result.
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// One pricing instance as the kernels see it.
struct Inst {
  double K, sigma, r, T, Smax, dS;
  int32_t Nx, P, Mf, Mg;
  int32_t C, NW, M, R, Np, Ws, pad0, pad1;  // partition of the tridiagonal rows
  int64_t coef_cn, coef_ie;    // offsets (doubles) of the two coefficient blocks in the pool
  int64_t exp_cn, exp_ie;      // offsets of exp(-r m dtau) tables (Mf+1 / Mg+1 entries)
  int64_t exp_sl;              // offset of exp(-r tau_n), n = 0..P (P+1 entries)
  int64_t state_off;           // offset of the instance in (P+1)*Nx arrays
  int64_t slice_off;           // offset of the instance in P*Nx arrays
  int64_t task_off;            // offset of the instance in per-slice arrays (P entries)
  int64_t task1_off;           // offset of the instance in per-boundary arrays (P+1 entries)
  int64_t norm_off;            // offset (pairs) in the norm partial sums: (P+1)*C pairs
};

// Coefficient block of one (instance, propagator): all doubles, GT global threads, Ws warps.
//   rows  [q][k][g], q: 0 lambda, 1 mu, 2 sigma, 3 alpha, 4 beta, 5 1/sigma
//   iface [q][g],    q: 0 kappa, 1 nu, 2 sigma_p, 3 1/sigma_p, 4 A, 5 C
//   pcr   [q][g],    q: 0..4 m1 per level, 5..9 m2 per level, 10 1/diag
//   resp  [q][g],    q: 0 response to Y_{w-1}, 1 response to Y_w
//   scr   [q][g],    q: set-up scratch (alpha, beta of the first and last inner row)
//   warp  [q][w],    q: 0 nu, 1 A, 2 C of the warp's lane 31
//   G     [Ws][Ws]   inverse of the cross-warp interface system
__host__ __device__ inline int64_t coef_rows_off(int q, int k, int g, int M, int GT) {
  return ((int64_t)q * M + k) * GT + g;
}
__host__ __device__ inline int64_t coef_if_off(int q, int g, int M, int GT) { return 6LL * M * GT + (int64_t)q * GT + g; }
__host__ __device__ inline int64_t coef_pcr_off(int q, int g, int M, int GT) {
  return 6LL * M * GT + 6LL * GT + (int64_t)q * GT + g;
}
__host__ __device__ inline int64_t coef_resp_off(int q, int g, int M, int GT) {
  return 6LL * M * GT + 17LL * GT + (int64_t)q * GT + g;
}
__host__ __device__ inline int64_t coef_scr_off(int q, int g, int M, int GT) {
  return 6LL * M * GT + 19LL * GT + (int64_t)q * GT + g;
}
__host__ __device__ inline int64_t coef_warp_off(int q, int w, int M, int GT, int Ws) {
  return 6LL * M * GT + 23LL * GT + (int64_t)q * Ws + w;
}
__host__ __device__ inline int64_t coef_G_off(int v, int u, int M, int GT, int Ws) {
  return 6LL * M * GT + 23LL * GT + 3LL * Ws + (int64_t)v * Ws + u;
}
__host__ __device__ inline int64_t coef_block_size(int M, int GT, int Ws) {
  return 6LL * M * GT + 23LL * GT + 3LL * Ws + (int64_t)Ws * Ws;
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
