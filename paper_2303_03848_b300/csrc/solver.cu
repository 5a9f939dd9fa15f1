// solver.cu -- Crank-Nicolson fine propagator, implicit Euler coarse
// propagator and the Parareal iteration (Eq. 7) on sm_103a.
//
// Section 3.2 of the paper: centred differences in S (Eq. 10), Crank-Nicolson
// for F and implicit Euler for G, both one tridiagonal solve per step.
//
// FP64 on this part issues one warp-wide DFMA per 64 cycles per SM
// sub-partition with a dependent-issue latency of the same length, so the
// cost of a step is the number of warp-level FP64 instructions it issues and
// the latency of whatever else sits on its critical path.  The design keeps
// the FP64 count near 5 per grid row per step:
//   * Crank-Nicolson is rewritten with Z = V^{m+1} + V^m:
//       (I - h L) Z = 2 V^m + boundary,  V^{m+1} = Z - V^m,  h = dtau/2,
//     and the state is carried scaled, W = 2 V / delta (delta = local LU
//     pivots), so the forward sweep needs no separate right-hand side product.
//   * Each thread eliminates its M-1 inner rows with a local Thomas sweep
//     (factorised once at set-up); the M-th row of every thread forms a
//     tridiagonal interface system that each warp reduces by parallel cyclic
//     reduction over shuffles (multipliers precomputed); the warps' lane-31
//     unknowns form a small system across the CTA -- or across a cluster of
//     CTAs that shares one grid over several SMs -- solved with a precomputed
//     inverse after one barrier per step.  A final fixup adds the interface
//     responses to the inner rows, or (coarse sweep, large clusters) a second
//     sweep over the inner rows with the interface values in place does the
//     same with fewer tables in shared memory.
// The whole grid stays in registers and shared memory for all steps of a slice.
#include <cooperative_groups.h>

#include <cmath>
#include <cstdio>

#include "bs_common.cuh"
#include "bs_internal.h"

namespace cg = cooperative_groups;

namespace bsp {

// ---------------------------------------------------------------------------
// Set-up: Eq. 10 coefficients, local LU factors, PCR multipliers, interface
// responses, cross-warp inverse and exp(-r m dtau) tables.
// ---------------------------------------------------------------------------

// Row r of (I - h L) in the partitioned layout (identity for padding and for
// the Dirichlet row at Smax).  Eq. 10 in tau with S_j = j dS:
//   a_j = sigma^2 j^2 / 2 - r j / 2, b_j = -sigma^2 j^2 - r, c_j = sigma^2 j^2 / 2 + r j / 2.
__device__ inline void mat_row(const Inst& in, double h, int r, double& l, double& d, double& u) {
  if (r < in.Np || r >= in.R - 1) {
    l = 0.0;
    d = 1.0;
    u = 0.0;
    return;
  }
  const int j = r - in.Np + 1;
  const double jj = (double)j, s2 = in.sigma * in.sigma;
  const double a = 0.5 * s2 * jj * jj - 0.5 * in.r * jj;
  const double b = -s2 * jj * jj - in.r;
  const double c = 0.5 * s2 * jj * jj + 0.5 * in.r * jj;
  l = (j == 1) ? 0.0 : -h * a;  // V_0 = 0 (Eq. 3) contributes nothing
  d = 1.0 - h * b;
  u = -h * c;
}

__device__ inline void kind_consts(const Inst& in, int kind, double& h, double& crhs, int& steps) {
  steps = kind == 0 ? in.Mf : in.Mg;
  const double dt = in.T / ((double)in.P * (double)steps);
  h = kind == 0 ? 0.5 * dt : dt;
  crhs = kind == 0 ? 2.0 : 1.0;
}

// Phase 1, one warp per (warp of the partition, instance): local LU of each
// thread's inner rows and their responses to the two neighbouring interfaces.
__global__ void __launch_bounds__(32) setup_rows_kernel(const Inst* insts, const int32_t* ids, double* pool,
                                                        double* exptab) {
  const Inst in = insts[ids[blockIdx.y]];
  const int w = blockIdx.x;
  if (w >= in.Ws) return;
  const int M = in.M, GT = in.Ws * 32;
  const int g = w * 32 + threadIdx.x;
  for (int kind = 0; kind < 2; ++kind) {
    double h, crhs;
    int steps;
    kind_consts(in, kind, h, crhs, steps);
    double* cb = pool + (kind == 0 ? in.coef_cn : in.coef_ie);
    if (w == 0) {
      double* et = exptab + (kind == 0 ? in.exp_cn : in.exp_ie);
      const double dt = in.T / ((double)in.P * (double)steps);
      for (int m = threadIdx.x; m <= steps; m += 32) et[m] = exp(-in.r * ((double)m * dt));
      if (kind == 0) {  // exp(-r tau_n) at the slice boundaries, tau_n = T n / P
        double* es = exptab + in.exp_sl;
        for (int n = threadIdx.x; n <= in.P; n += 32) es[n] = exp(-in.r * (in.T * (double)n / (double)in.P));
      }
    }
    double lam[32], mu[32], del[32];
    double prev_u = 0.0;
    for (int k = 0; k < M - 1; ++k) {
      const int r = g * M + k;
      double l, d, u;
      mat_row(in, h, r, l, d, u);
      del[k] = (k == 0) ? d : d - l * (prev_u / del[k - 1]);
      lam[k] = l / del[k];
      mu[k] = u / del[k];
      prev_u = u;
      const bool pad = r < in.Np;
      cb[coef_rows_off(0, k, g, M, GT)] = lam[k];
      cb[coef_rows_off(1, k, g, M, GT)] = mu[k];
      cb[coef_rows_off(2, k, g, M, GT)] = pad ? 0.0 : crhs / del[k];
      cb[coef_rows_off(5, k, g, M, GT)] = pad ? 0.0 : del[k] / crhs;
    }
    double phi[32];
    phi[0] = -lam[0];
    for (int k = 1; k < M - 1; ++k) phi[k] = -lam[k] * phi[k - 1];
    double alp = phi[M - 2], bet = -mu[M - 2];
    cb[coef_rows_off(3, M - 2, g, M, GT)] = alp;
    cb[coef_rows_off(4, M - 2, g, M, GT)] = bet;
    cb[coef_scr_off(2, g, M, GT)] = alp;
    cb[coef_scr_off(3, g, M, GT)] = bet;
    for (int k = M - 3; k >= 0; --k) {
      alp = phi[k] - mu[k] * alp;
      bet = -mu[k] * bet;
      cb[coef_rows_off(3, k, g, M, GT)] = alp;
      cb[coef_rows_off(4, k, g, M, GT)] = bet;
    }
    cb[coef_scr_off(0, g, M, GT)] = alp;
    cb[coef_scr_off(1, g, M, GT)] = bet;
    for (int q = 0; q < 6; ++q) cb[coef_rows_off(q, M - 1, g, M, GT)] = 0.0;  // interface row slots unused
  }
}

// Phase 2: interface rows, in-warp PCR multipliers and responses.
__global__ void __launch_bounds__(32) setup_iface_kernel(const Inst* insts, const int32_t* ids, double* pool) {
  const Inst in = insts[ids[blockIdx.y]];
  const int w = blockIdx.x;
  if (w >= in.Ws) return;
  const int M = in.M, GT = in.Ws * 32, Ws = in.Ws;
  const int L = threadIdx.x, g = w * 32 + L;
  for (int kind = 0; kind < 2; ++kind) {
    double h, crhs;
    int steps;
    kind_consts(in, kind, h, crhs, steps);
    double* cb = pool + (kind == 0 ? in.coef_cn : in.coef_ie);
    double A = 0.0, C = 0.0, kap = 0.0, nu = 0.0, sigp = 0.0, isigp = 0.0;
    if (g < GT - 1) {
      // interface row p: l x_{p-1} + d x_p + u x_{p+1} = r_p with the inner
      // neighbours written through their interface responses, divided by D
      const int p = g * M + M - 1;
      double l, d, u;
      mat_row(in, h, p, l, d, u);
      const double a_last = cb[coef_scr_off(2, g, M, GT)], b_last = cb[coef_scr_off(3, g, M, GT)];
      const double a_next = cb[coef_scr_off(0, g + 1, M, GT)], b_next = cb[coef_scr_off(1, g + 1, M, GT)];
      const double D = d + l * b_last + u * a_next;
      A = l * a_last / D;
      C = u * b_next / D;
      kap = l / D;
      nu = u / D;
      const bool pad = p < in.Np;
      sigp = pad ? 0.0 : crhs / D;
      isigp = pad ? 0.0 : D / crhs;
    }
    cb[coef_if_off(0, g, M, GT)] = kap;
    cb[coef_if_off(1, g, M, GT)] = nu;
    cb[coef_if_off(2, g, M, GT)] = sigp;
    cb[coef_if_off(3, g, M, GT)] = isigp;
    cb[coef_if_off(4, g, M, GT)] = A;
    cb[coef_if_off(5, g, M, GT)] = C;
    if (L == 31) {
      cb[coef_warp_off(0, w, M, GT, Ws)] = nu;
      cb[coef_warp_off(1, w, M, GT, Ws)] = A;
      cb[coef_warp_off(2, w, M, GT, Ws)] = C;
    }
    // PCR multipliers of the in-warp interface system with zero external
    // couplings (lane 31 is the warp's cross-warp unknown, solved separately).
    double a_ = (L == 0 || L == 31) ? 0.0 : A;
    double c_ = (L >= 30) ? 0.0 : C;
    double d_ = 1.0;
    double m1[kPcrLevels], m2[kPcrLevels];
#pragma unroll
    for (int lv = 0; lv < kPcrLevels; ++lv) {
      const int s = 1 << lv;
      const double aU = __shfl_up_sync(kFull, a_, s), cU = __shfl_up_sync(kFull, c_, s),
                   dU = __shfl_up_sync(kFull, d_, s);
      const double aD = __shfl_down_sync(kFull, a_, s), cD = __shfl_down_sync(kFull, c_, s),
                   dD = __shfl_down_sync(kFull, d_, s);
      const bool vu = L >= s, vd = L + s < 32;
      const double k1 = vu ? a_ / dU : 0.0;
      const double k2 = vd ? c_ / dD : 0.0;
      const double na = vu ? -k1 * aU : 0.0;
      const double nc = vd ? -k2 * cD : 0.0;
      const double nd = d_ - (vu ? k1 * cU : 0.0) - (vd ? k2 * aD : 0.0);
      a_ = na;
      c_ = nc;
      d_ = nd;
      m1[lv] = k1;
      m2[lv] = k2;
      cb[coef_pcr_off(lv, g, M, GT)] = k1;
      cb[coef_pcr_off(5 + lv, g, M, GT)] = k2;
    }
    const double inv = 1.0 / d_;
    cb[coef_pcr_off(10, g, M, GT)] = inv;
    // responses of lanes 0..30 to Y_{w-1} (enters lane 0 as -A) and Y_w
    // (enters lane 30 as -C), with the same recursion the step uses
    double ea = (L == 0) ? -A : 0.0, ec = (L == 30) ? -C : 0.0;
#pragma unroll
    for (int lv = 0; lv < kPcrLevels; ++lv) {
      const int s = 1 << lv;
      const double ua = __shfl_up_sync(kFull, ea, s), da = __shfl_down_sync(kFull, ea, s);
      const double uc = __shfl_up_sync(kFull, ec, s), dc = __shfl_down_sync(kFull, ec, s);
      ea = fma(-m1[lv], ua, fma(-m2[lv], da, ea));
      ec = fma(-m1[lv], uc, fma(-m2[lv], dc, ec));
    }
    cb[coef_resp_off(0, g, M, GT)] = (L == 31) ? 0.0 : ea * inv;
    cb[coef_resp_off(1, g, M, GT)] = (L == 31) ? 0.0 : ec * inv;
  }
}

// Phase 3, one CTA per (instance, propagator): the cross-warp system over
// Y_w = X at lane 31 of warp w (Y_{Ws-1} is the Dirichlet row) and its inverse
// by Gauss-Jordan with partial pivoting.
__global__ void __launch_bounds__(128) setup_cross_kernel(const Inst* insts, const int32_t* ids, double* pool) {
  extern __shared__ double mx_raw[];
  __shared__ int s_piv;
  const Inst in = insts[ids[blockIdx.x]];
  const int kind = blockIdx.y;
  const int M = in.M, GT = in.Ws * 32, Ws = in.Ws;
  const int ld = 2 * Ws + 1;
  auto Mx = [&](int i) -> double* { return mx_raw + (size_t)i * ld; };
  double* cb = pool + (kind == 0 ? in.coef_cn : in.coef_ie);
  const int t = threadIdx.x;
  for (int e = t; e < Ws * 2 * Ws; e += blockDim.x) {
    const int i = e / (2 * Ws), j = e % (2 * Ws);
    Mx(i)[j] = (j == Ws + i) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int w = t; w < Ws; w += blockDim.x) {
    if (w == Ws - 1) {
      Mx(w)[w] = 1.0;
      continue;
    }
    const int t30 = 32 * w + 30, tn0 = 32 * (w + 1);
    const double A31 = cb[coef_warp_off(1, w, M, GT, Ws)], C31 = cb[coef_warp_off(2, w, M, GT, Ws)];
    const double ra30 = cb[coef_resp_off(0, t30, M, GT)], rc30 = cb[coef_resp_off(1, t30, M, GT)];
    const double ra0 = cb[coef_resp_off(0, tn0, M, GT)], rc0 = cb[coef_resp_off(1, tn0, M, GT)];
    if (w > 0) Mx(w)[w - 1] = A31 * ra30;
    Mx(w)[w] = 1.0 + A31 * rc30 + C31 * ra0;
    Mx(w)[w + 1] = C31 * rc0;
  }
  __syncthreads();
  for (int c = 0; c < Ws; ++c) {
    if (t == 0) {
      int piv = c;
      for (int i = c + 1; i < Ws; ++i)
        if (fabs(Mx(i)[c]) > fabs(Mx(piv)[c])) piv = i;
      s_piv = piv;
    }
    __syncthreads();
    const int piv = s_piv;
    if (piv != c)
      for (int j = t; j < 2 * Ws; j += blockDim.x) {
        const double tmp = Mx(c)[j];
        Mx(c)[j] = Mx(piv)[j];
        Mx(piv)[j] = tmp;
      }
    __syncthreads();
    const double ip = 1.0 / Mx(c)[c];
    __syncthreads();
    for (int j = t; j < 2 * Ws; j += blockDim.x) Mx(c)[j] *= ip;
    __syncthreads();
    for (int e = t; e < Ws * 2 * Ws; e += blockDim.x) {
      const int i = e / (2 * Ws), j = e % (2 * Ws);
      if (i != c && j != c) Mx(i)[j] -= Mx(i)[c] * Mx(c)[j];
    }
    __syncthreads();
    for (int i = t; i < Ws; i += blockDim.x)
      if (i != c) Mx(i)[c] = 0.0;
    __syncthreads();
  }
  for (int e = t; e < Ws * Ws; e += blockDim.x) {
    const int v = e / Ws, u = e % Ws;
    cb[coef_G_off(v, u, M, GT, Ws)] = Mx(v)[Ws + u];
  }
}

// ---------------------------------------------------------------------------
// One time step of the partitioned solver.
// ---------------------------------------------------------------------------

// A step can finish by sweeping the inner rows again with the interface
// values in place (2 FMA per row, the same count as adding the precomputed
// interface responses), which needs only 3 coefficient tables (24 bytes per
// row) in shared memory instead of 5.  The fine propagation does so on
// clusters of 8 or more CTAs with 4 or more rows per thread, where the smaller
// tables let 8-CTA clusters of 8-warp CTAs hold grids that took 16-CTA
// clusters; the coarse sweep always does (twice the instances per SM).
template <int M, int C>
__host__ __device__ constexpr bool resweep_class() {
  return C >= 8 && M >= 4;
}

// S2 slices share one CTA (and its tables): thread group g = threadIdx.x / T runs
// its own slice of the same instance with its own exchange buffers.
template <int M, int NW, int C, int S2 = 1, bool RS = resweep_class<M, C>()>
struct SolverSmem {
  static constexpr int T = NW * 32, Ws = C * NW;
  static constexpr int kTabs = RS ? 3 : 5;
  double rows[kTabs][M][T];  // lambda, mu, sigma (and alpha, beta) of the group's threads
  double G2[NW][2][Ws];     // rows w-1 and w of the cross-warp inverse, per local warp
  double nu31[Ws], A31[Ws], C31[Ws];
  alignas(16) double pub[S2][2][Ws][4];  // [group][step parity][global warp][x0, X0, X30, R31]
  double red[S2][2][NW];
  alignas(8) unsigned long long bar[S2][2];  // C > 1: arrival of a step's values, per group and parity
};

// Thread index within its slice group and the group index.
template <int NW>
__device__ __forceinline__ int lthread() {
  return (int)threadIdx.x % (NW * 32);
}
template <int NW>
__device__ __forceinline__ int lgroup() {
  return (int)threadIdx.x / (NW * 32);
}

struct SolverRegs {
  double kap, nu, sigp, isigp;
  double m1[kPcrLevels], m2[kPcrLevels], inv, ra, rc;
  double mlast;  // the last PCR level's one multiplier (lanes 0-15 couple up, 16-31 down)
  // M = 2: the step's state update written as K + e Y_{w-1} + f Y_w per row, with
  // K formed before the cross-warp unknowns arrive (see step_finish)
  double s0, sa, sb, e0, f0, sp, g1, h1;
  int fail;  // a bounded wait gave up (sticky; later waits are skipped)
};

// Clusters exchange the per-step values with st.async into every CTA's
// buffer, each store completing transaction bytes on the receiver's mbarrier:
// one point-to-point arrival per step instead of a cluster-wide barrier.
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t cluster_addr(uint32_t a, int rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}

__device__ __forceinline__ void mbar_init(uint32_t a) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(a) : "memory");
}

__device__ __forceinline__ void mbar_expect(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}

__device__ __forceinline__ void st_async2(uint32_t raddr, double v0, double v1, uint32_t rbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f64 [%0], {%1, %2}, [%3];" ::"r"(raddr),
               "d"(v0), "d"(v1), "r"(rbar)
               : "memory");
}

// Wait for phase parity ph of the mbarrier at a, at most about 2^31 cycles (one
// second); false when the limit was reached.
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t ph) {
  const long long t0 = clock64();
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(ph)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > (1ll << 31)) return false;
  }
}

template <int C>
__device__ __forceinline__ int cta_rank() {
  if constexpr (C == 1) {
    return 0;
  } else {
    return (int)cg::this_cluster().block_rank();
  }
}

template <int M, int NW, int C, int S2 = 1, bool RS = resweep_class<M, C>()>
__device__ __forceinline__ void load_solver(const double* __restrict__ cb, SolverSmem<M, NW, C, S2, RS>& sm,
                                            SolverRegs& rg) {
  constexpr int T = NW * 32, Ws = C * NW, GT = C * T;
  const int t = lthread<NW>(), c = cta_rank<C>();  // both groups write the same table entries
  const int g = c * T + t;
  for (int q = 0; q < SolverSmem<M, NW, C, S2, RS>::kTabs; ++q)
    for (int k = 0; k < M; ++k) sm.rows[q][k][t] = cb[coef_rows_off(q, k, g, M, GT)];
  rg.kap = cb[coef_if_off(0, g, M, GT)];
  rg.nu = cb[coef_if_off(1, g, M, GT)];
  rg.sigp = cb[coef_if_off(2, g, M, GT)];
  rg.isigp = cb[coef_if_off(3, g, M, GT)];
#pragma unroll
  for (int lv = 0; lv < kPcrLevels; ++lv) {
    rg.m1[lv] = cb[coef_pcr_off(lv, g, M, GT)];
    rg.m2[lv] = cb[coef_pcr_off(5 + lv, g, M, GT)];
  }
  rg.inv = cb[coef_pcr_off(10, g, M, GT)];
  rg.mlast = (t & 31) < 16 ? rg.m2[kPcrLevels - 1] : rg.m1[kPcrLevels - 1];
  rg.ra = cb[coef_resp_off(0, g, M, GT)];
  rg.rc = cb[coef_resp_off(1, g, M, GT)];
  if constexpr (M == 2) {
    // X = Xt + ra Yl + rc Yr on lanes 0..30 and X = Yr on lane 31; the inner
    // row's left neighbour is the previous lane's X (Yl on lane 0)
    const int L = t & 31;
    const double ra = L == 31 ? 0.0 : rg.ra, rc = L == 31 ? 1.0 : rg.rc;
    double rap = __shfl_up_sync(kFull, ra, 1), rcp = __shfl_up_sync(kFull, rc, 1);
    if (L == 0) {
      rap = 1.0;
      rcp = 0.0;
    }
    const double s0 = cb[coef_rows_off(2, 0, g, M, GT)];
    const double al = cb[coef_rows_off(3, 0, g, M, GT)], be = cb[coef_rows_off(4, 0, g, M, GT)];
    // the step hands on PCR's result before its scaling by inv (see step_reduce):
    // the users of a lane's Xt take that lane's inv in their coefficients
    const double inv_prev = __shfl_up_sync(kFull, rg.inv, 1);
    rg.s0 = s0;
    rg.sa = L == 0 ? 0.0 : s0 * al * inv_prev;
    rg.sb = L == 31 ? 0.0 : s0 * be * rg.inv;
    rg.e0 = s0 * (al * rap + be * ra);
    rg.f0 = s0 * (al * rcp + be * rc);
    rg.sp = L == 31 ? 0.0 : rg.sigp * rg.inv;
    rg.g1 = rg.sigp * ra;
    rg.h1 = rg.sigp * rc;
  }
  for (int i = t; i < Ws; i += T) {
    sm.nu31[i] = cb[coef_warp_off(0, i, M, GT, Ws)];
    sm.A31[i] = cb[coef_warp_off(1, i, M, GT, Ws)];
    sm.C31[i] = cb[coef_warp_off(2, i, M, GT, Ws)];
    if constexpr (M == 2) {  // published X30 and X0 unscaled (lane 30 of warp i, lane 0 of warp i + 1)
      sm.A31[i] *= cb[coef_pcr_off(10, 32 * i + 30, M, GT)];
      if (i + 1 < Ws) sm.C31[i] *= cb[coef_pcr_off(10, 32 * (i + 1), M, GT)];
    }
  }
  for (int i = t; i < NW * 2 * Ws; i += T) {
    const int wl = i / (2 * Ws), side = (i / Ws) % 2, u = i % Ws;
    const int row = c * NW + wl - 1 + side;  // global warp w-1 (side 0) or w (side 1)
    sm.G2[wl][side][u] = row >= 0 ? cb[coef_G_off(row, u, M, GT, Ws)] : 0.0;
  }
  __syncthreads();  // the kernel's cluster barrier follows before any exchange
}

// The exchange barriers, once per launch (a cluster barrier follows before the
// first step; the step counter then runs on across slices and tasks).
template <int M, int NW, int C, int S2 = 1, bool RS = resweep_class<M, C>()>
__device__ __forceinline__ void exchange_init(SolverSmem<M, NW, C, S2, RS>& sm, SolverRegs& rg) {
  rg.fail = 0;
  if (C > 1 && threadIdx.x == 0) {
    for (int g = 0; g < S2; ++g) {
      mbar_init(smem_addr(&sm.bar[g][0]));
      mbar_init(smem_addr(&sm.bar[g][1]));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
}

// A CTA whose wait gave up records BS_TIMEOUT and waits (again bounded) for the
// values of the last two steps that may still be arriving in its buffers.
template <int M, int NW, int C, int S2 = 1, bool RS = resweep_class<M, C>()>
__device__ __forceinline__ void exchange_drain(SolverSmem<M, NW, C, S2, RS>& sm, const SolverRegs& rg, int seq,
                                               int* status) {
  if constexpr (C > 1) {
    if (!rg.fail) return;
    const int gi = lgroup<NW>();
    for (int q = seq - 2; q < seq; ++q)
      if (q >= 0) (void)mbar_wait(smem_addr(&sm.bar[gi][q & 1]), (uint32_t)(q >> 1) & 1u);
    if (status != nullptr && lthread<NW>() == 0) atomicExch(status, 6);  // BS_TIMEOUT
  }
}

// One step in two halves around the barrier.  step_reduce: local sweeps,
// interface right-hand side, in-warp PCR, publication of the warp's boundary
// values, barrier arrival.  step_finish: barrier wait, cross-warp unknowns,
// interface values, fixup of the inner rows and the scaled state update.
// x receives the solution of the step (Z for Crank-Nicolson, V^{m+1} for
// implicit Euler) on the thread's rows; W is advanced to the next scaled state.
// Zb is the Dirichlet value of the step (used by the grid's last thread).
template <int M, int NW, int C, int S2 = 1, bool RS = resweep_class<M, C>()>
__device__ __forceinline__ double step_reduce(const double (&W)[M], double (&x)[M], SolverSmem<M, NW, C, S2, RS>& sm,
                                              const SolverRegs& rg, double Zb, int seq) {
  const int par = seq & 1;
  constexpr int Ws = C * NW;
  const int t = lthread<NW>(), L = t & 31, wl = t >> 5, gi = lgroup<NW>();
  const int c = cta_rank<C>();
  const int w = c * NW + wl;
  // 1. local forward and backward sweeps over the inner rows (zero interfaces)
  x[0] = W[0];
#pragma unroll
  for (int k = 1; k <= M - 2; ++k) x[k] = fma(-sm.rows[0][k][t], x[k - 1], W[k]);
#pragma unroll
  for (int k = M - 3; k >= 0; --k) x[k] = fma(-sm.rows[1][k][t], x[k + 1], x[k]);
  // 2. interface right-hand side; lane 31 completes its term with the next
  //    warp's first inner value after the barrier
  const double xs_next = __shfl_down_sync(kFull, x[0], 1);
  double R = fma(-rg.kap, x[M - 2], W[M - 1]);
  if (L != 31) R = fma(-rg.nu, xs_next, R);
  if (w == Ws - 1 && L == 31) R = Zb;  // Dirichlet row at Smax
  // 3. in-warp PCR on lanes 0..30 with zero external couplings
  double Rp = (L == 31) ? 0.0 : R;
#pragma unroll
  for (int lv = 0; lv < kPcrLevels - 1; ++lv) {
    const int s = 1 << lv;
    const double up = __shfl_up_sync(kFull, Rp, s);
    const double dn = __shfl_down_sync(kFull, Rp, s);
    Rp = fma(-rg.m1[lv], up, fma(-rg.m2[lv], dn, Rp));
  }
  // stride 16: lane L couples to lane L ^ 16 only (the set-up zeroes the other
  // multiplier), so one exchange and one FMA do what the two-sided level does
  Rp = fma(-rg.mlast, __shfl_xor_sync(kFull, Rp, 16), Rp);
  // M = 2 folds the scaling by inv into the coefficients that use Xt (its own
  // state update and the cross-warp solve), one FP64 instruction fewer per step
  const double Xt = (M == 2) ? Rp : Rp * rg.inv;
  // 4. publish this warp's boundary values to every CTA of the grid
  const double p0 = __shfl_sync(kFull, x[0], 0);
  const double p1 = __shfl_sync(kFull, Xt, 0);
  const double p2 = __shfl_sync(kFull, Xt, 30);
  const double p3 = __shfl_sync(kFull, R, 31);
  if constexpr (C == 1) {
    if (L == 0) {
      sm.pub[gi][par][w][0] = p0;
      sm.pub[gi][par][w][1] = p1;
      sm.pub[gi][par][w][2] = p2;
      sm.pub[gi][par][w][3] = p3;
    }
  } else {
    // this CTA expects 32 bytes from every warp of the grid; lane L sends this
    // warp's 32 bytes to CTA L
    if (t == 0) mbar_expect(smem_addr(&sm.bar[gi][par]), (uint32_t)Ws * 32u);
    if (L < C) {
      const uint32_t slot = cluster_addr(smem_addr(&sm.pub[gi][par][w][0]), L);
      const uint32_t rbar = cluster_addr(smem_addr(&sm.bar[gi][par]), L);
      st_async2(slot, p0, p1, rbar);
      st_async2(slot + 16u, p2, p3, rbar);
    }
  }
  return Xt;
}

template <int M, int NW, int C, bool CN, int S2 = 1, bool RS = resweep_class<M, C>()>
__device__ __forceinline__ void step_finish(double (&W)[M], double (&x)[M], SolverSmem<M, NW, C, S2, RS>& sm,
                                            SolverRegs& rg, double Xt, int seq) {
  const int par = seq & 1;
  constexpr int Ws = C * NW;
  constexpr bool kHalves = Ws <= 16;  // lanes 0-15 form Y_{w-1}, lanes 16-31 Y_w
  constexpr int NU = kHalves ? 1 : (Ws + 31) / 32;
  const int t = lthread<NW>(), L = t & 31, wl = t >> 5, gi = lgroup<NW>();
  auto& pub = sm.pub[gi];
  // constants of the cross-warp solve for the lanes' warps u, read while the
  // other CTAs' values arrive
  double cnu[NU], ca[NU], cc[NU], g0[NU], g1[NU];
#pragma unroll
  for (int q = 0; q < NU; ++q) {
    const int u = kHalves ? (L & 15) : q * 32 + L;
    const bool ok = u < Ws;
    cnu[q] = ok ? sm.nu31[u] : 0.0;
    ca[q] = ok ? sm.A31[u] : 0.0;
    cc[q] = ok ? sm.C31[u] : 0.0;
    g0[q] = ok ? sm.G2[wl][kHalves ? (L >> 4) : 0][u] : 0.0;
    g1[q] = ok ? sm.G2[wl][1][u] : 0.0;
  }
  // M = 2, the part of the state update that does not depend on the
  // cross-warp unknowns (formed while they arrive):
  //   W_0' = [s0 x_0 - W_0 + s0 al Xt_{L-1} + s0 be Xt] + e0 Y_{w-1} + f0 Y_w,
  //   W_1' = [sigp Xt - W_1] + g1 Y_{w-1} + h1 Y_w   (no -W terms for implicit Euler)
  double K0 = 0.0, K1 = 0.0;
  if constexpr (M == 2) {
    const double Xtp = __shfl_up_sync(kFull, Xt, 1);
    K0 = fma(rg.sa, Xtp, fma(rg.sb, Xt, CN ? fma(rg.s0, x[0], -W[0]) : rg.s0 * x[0]));
    K1 = CN ? fma(rg.sp, Xt, -W[1]) : rg.sp * Xt;
  }
  if constexpr (C == 1 && S2 == 1) {
    __syncthreads();
  } else if constexpr (C == 1) {
    // slice pairs in one CTA: each group waits on its own named barrier (ids 1
    // and 2; 0 is the block barrier), so a group whose slice is inactive
    // takes no step barrier at all
    if (gi == 0) {
      asm volatile("bar.sync 1, %0;" ::"n"(NW * 32) : "memory");
    } else {
      asm volatile("bar.sync 2, %0;" ::"n"(NW * 32) : "memory");
    }
  } else {
    if (!rg.fail && !mbar_wait(smem_addr(&sm.bar[gi][par]), (uint32_t)(seq >> 1) & 1u)) rg.fail = 1;
  }
  // 5. cross-warp unknowns: rho_u by lane u, then Y_{w-1} and Y_w as dot
  //    products with rows of the precomputed inverse
  double Yl, Yr;
  if constexpr (kHalves) {
    const int u = L & 15;
    double v = 0.0;
    if (u < Ws) {
      double rho;
      if (u == Ws - 1) {
        rho = pub[par][u][3];
      } else {
        rho = fma(-cnu[0], pub[par][u + 1][0], pub[par][u][3]);
        rho = fma(-ca[0], pub[par][u][2], rho);
        rho = fma(-cc[0], pub[par][u + 1][1], rho);
      }
      v = g0[0] * rho;
    }
#pragma unroll
    for (int s = 1; s < Ws; s <<= 1) v += __shfl_xor_sync(kFull, v, s);
    Yl = __shfl_sync(kFull, v, 0);
    Yr = __shfl_sync(kFull, v, 16);
  } else {
    double pl = 0.0, pr = 0.0;
#pragma unroll
    for (int q = 0; q < NU; ++q) {
      const int u = q * 32 + L;
      if (u < Ws) {
        double rho;
        if (u == Ws - 1) {
          rho = pub[par][u][3];
        } else {
          rho = fma(-cnu[q], pub[par][u + 1][0], pub[par][u][3]);
          rho = fma(-ca[q], pub[par][u][2], rho);
          rho = fma(-cc[q], pub[par][u + 1][1], rho);
        }
        pl = fma(g0[q], rho, pl);
        pr = fma(g1[q], rho, pr);
      }
    }
    // reduce-scatter of the two sums: the first level leaves the Y_{w-1} partial
    // on even lanes and the Y_w partial on odd lanes, then one sum per level
    const bool odd = (L & 1) != 0;
    double v = (odd ? pr : pl) + __shfl_xor_sync(kFull, odd ? pl : pr, 1);
#pragma unroll
    for (int s = 2; s < 32; s <<= 1) v += __shfl_xor_sync(kFull, v, s);
    Yl = __shfl_sync(kFull, v, 0);
    Yr = __shfl_sync(kFull, v, 1);
  }
  if constexpr (M == 2) {
    // 6. scaled state update from the pre-formed parts
    W[0] = fma(rg.e0, Yl, fma(rg.f0, Yr, K0));
    W[1] = fma(rg.g1, Yl, fma(rg.h1, Yr, K1));
  } else {
    const double X = (L == 31) ? Yr : fma(rg.rc, Yr, fma(rg.ra, Yl, Xt));
    double Xprev = __shfl_up_sync(kFull, X, 1);
    if (L == 0) Xprev = Yl;
    if constexpr (RS) {
      // 6. the inner rows swept again with the interface values in place: the
      //    forward sweep from X_{g-1} (coupled to the first inner row through
      //    lambda_0), the back substitution from X_g (coupled to the last one
      //    through mu_{M-2}); then the scaled state update
      x[0] = fma(-sm.rows[0][0][t], Xprev, W[0]);
#pragma unroll
      for (int k = 1; k <= M - 2; ++k) x[k] = fma(-sm.rows[0][k][t], x[k - 1], W[k]);
#pragma unroll
      for (int k = M - 2; k >= 0; --k) {
        x[k] = fma(-sm.rows[1][k][t], k == M - 2 ? X : x[k + 1], x[k]);
        W[k] = CN ? fma(sm.rows[2][k][t], x[k], -W[k]) : sm.rows[2][k][t] * x[k];
      }
    } else {
      // 6. fixup of the inner rows and the scaled state update
#pragma unroll
      for (int k = 0; k <= M - 2; ++k) {
        const double xv = fma(sm.rows[4][k][t], X, fma(sm.rows[3][k][t], Xprev, x[k]));
        x[k] = xv;
        W[k] = CN ? fma(sm.rows[2][k][t], xv, -W[k]) : sm.rows[2][k][t] * xv;
      }
    }
    x[M - 1] = X;
    W[M - 1] = CN ? fma(rg.sigp, X, -W[M - 1]) : rg.sigp * X;
  }
}

// Read the Nx-vector V into the thread's rows and scale it into W.
template <int M, int NW, int C, int S2 = 1, bool RS = resweep_class<M, C>()>
__device__ __forceinline__ void load_state(const Inst& in, const double* __restrict__ V,
                                           const SolverSmem<M, NW, C, S2, RS>& sm, const SolverRegs& rg, double (&W)[M]) {
  const int t = lthread<NW>(), g = cta_rank<C>() * NW * 32 + t;
#pragma unroll
  for (int k = 0; k < M; ++k) {
    const int j = g * M + k - in.Np + 1;
    const double v = (j >= 1 && j <= in.Nx - 2) ? V[j] : 0.0;
    W[k] = (k < M - 1) ? sm.rows[2][k][t] * v : rg.sigp * v;
  }
}

// Value of row k of this thread after a slice, V = W / sigma (the scaled state
// of both propagators: W = 2V/delta-scaled for Crank-Nicolson, sigma x for
// implicit Euler).
template <int M, int NW, int C, bool CN>
__device__ __forceinline__ double row_value(const double* __restrict__ cb, int k, const double (&W)[M],
                                            const double (&x)[M], double isigp) {
  (void)x;
  const int g = cta_rank<C>() * NW * 32 + lthread<NW>();
  const double is = (k < M - 1) ? cb[coef_rows_off(5, k, g, M, C * NW * 32)] : isigp;
  return W[k] * is;
}

// Run `steps` steps of the propagator on slice n starting from scaled state W.
// The right Dirichlet value of the next step is formed while the barrier
// completes, from exp(-r m dtau) read one step ahead; KeN = K exp(-r tau_n) of
// the slice's start (slice_KeN, or from the set-up table of exp(-r tau_n)).
template <int M, int NW, int C, bool CN, int S2 = 1, bool RS = resweep_class<M, C>()>
__device__ __forceinline__ void run_slice(const Inst& in, double KeN, const double* __restrict__ et, int steps,
                                          double (&W)[M], double (&x)[M], SolverSmem<M, NW, C, S2, RS>& sm,
                                          SolverRegs& rg, int& seq) {
  const bool last_warp = cta_rank<C>() == C - 1 && (lthread<NW>() >> 5) == NW - 1;
  double Bold = in.Smax - KeN;  // exp(0) = 1
  double Zb = 0.0, e_next = 0.0;
  if (last_warp) {
    const double Bnew = fma(-KeN, __ldg(et + 1), in.Smax);
    Zb = CN ? Bold + Bnew : Bnew;
    Bold = Bnew;
    if (steps >= 2) e_next = __ldg(et + 2);
  }
  for (int m = 0; m < steps; ++m) {
    const double Xt = step_reduce<M, NW, C, S2>(W, x, sm, rg, Zb, seq);
    if (last_warp) {  // Dirichlet value of step m + 1 (unused after the last step)
      const double Bnew = fma(-KeN, e_next, in.Smax);
      Zb = CN ? Bold + Bnew : Bnew;
      Bold = Bnew;
      if (m + 3 <= steps) e_next = __ldg(et + m + 3);
    }
    step_finish<M, NW, C, CN, S2>(W, x, sm, rg, Xt, seq);
    ++seq;
  }
}

// Sum of two doubles over a slice group's NW warps, result valid on the
// group's thread 0.  Contains CTA-wide barriers: every thread of the CTA calls it.
template <int NW>
__device__ __forceinline__ void block_sum2(double& a, double& b, double (*red)[NW]) {
  const int t = lthread<NW>(), L = t & 31, w = t >> 5;
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    a += __shfl_down_sync(kFull, a, s);
    b += __shfl_down_sync(kFull, b, s);
  }
  __syncthreads();
  if (L == 0) {
    red[0][w] = a;
    red[1][w] = b;
  }
  __syncthreads();
  if (t == 0) {
    for (int i = 1; i < NW; ++i) {
      a += red[0][i];
      b += red[1][i];
    }
  }
}

__device__ __forceinline__ double bc_right(const Inst& in, int n) {
  return in.Smax - in.K * exp(-in.r * (in.T * (double)n / (double)in.P));
}

// The same from the set-up table es[n] = exp(-r tau_n) (bitwise the same value):
// the kernels that take one step per slice use it and compute no exponential.
__device__ __forceinline__ double bc_right(const Inst& in, const double* __restrict__ es, int n) {
  return in.Smax - in.K * es[n];
}

__device__ __forceinline__ double slice_KeN(const Inst& in, int n) {
  const double tau_n = in.T * (double)n / (double)in.P;
  return in.K * exp(-in.r * tau_n);
}

// ---------------------------------------------------------------------------
// Propagation over slices: fine (Crank-Nicolson) or coarse (implicit Euler).
// One cluster of C CTAs per (instance, slice): blockIdx.x = slice * C + rank.
// ---------------------------------------------------------------------------

template <int M, int NW, int C, bool CN, int S2>
__global__ void __launch_bounds__(S2 * NW * 32, 1) prop_kernel(PropArgs a) {
  constexpr int T = NW * 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_task;
  // every instance has converged: nothing to do (the same value for every CTA)
  if (a.n_live != nullptr && *a.n_live == 0) return;
  // implicit Euler (coarse_propagate, the network-anchored corrections) takes
  // the coarse sweep's re-sweep finish, so the two give the same values bit for bit
  constexpr bool RS = CN ? resweep_class<M, C>() : true;
  SolverSmem<M, NW, C, S2, RS>& sm = *reinterpret_cast<SolverSmem<M, NW, C, S2, RS>*>(smem_raw);
  const int t = lthread<NW>(), gi = lgroup<NW>(), c = cta_rank<C>();
  SolverRegs rg;
  exchange_init<M, NW, C, S2>(sm, rg);
  int seq = 0;
  // persistent: a task group is S2 consecutive slices of one instance from
  // slice kb = max(k_iter, 0) on (group gi takes slice kb + S2 j + gi), so at
  // most one group per instance is half idle.  Clusters walk the task groups
  // q, q + clusters, ...; one-CTA grids given a counter take the next group
  // from it, which balances the load when slices before kb or instances that
  // have converged leave some groups empty.  Skipping a whole group is uniform
  // over the cluster; a group whose own slice is inactive still takes every
  // block and cluster barrier.
  const int kb = a.k_iter > 0 ? a.k_iter : 0;
  const int ngrp = (a.maxP - kb + S2 - 1) / S2;
  const int64_t n_cl = gridDim.x / C, ntask = (int64_t)a.n_inst * ngrp;
  const bool dyn = C == 1 && a.task_ctr != nullptr;
  auto grab = [&]() -> int64_t {  // every thread of the CTA calls it
    __syncthreads();              // all threads have read the previous value
    if (threadIdx.x == 0) s_task = atomicAdd(a.task_ctr, 1);
    __syncthreads();
    return (int64_t)s_task;
  };
  for (int64_t task = dyn ? grab() : blockIdx.x / C; task < ntask; task = dyn ? grab() : task + n_cl) {
    const int idx = a.ids[task / ngrp];
    const int n0 = kb + (int)(task % ngrp) * S2;
    const Inst in = a.insts[idx];
    auto live = [&](int n) {
      if (n >= in.P) return false;
      if (a.k_iter >= 0 && n < a.k_iter) return false;
      if (a.ctrl != nullptr && a.ctrl[idx].done) return false;
      if (a.active != nullptr && !a.active[in.task_off + n]) return false;
      return true;
    };
    bool any = false;
#pragma unroll
    for (int g = 0; g < S2; ++g) any = any || live(n0 + g);
    if (!any) continue;
    const int n = n0 + gi;
    const bool mine = live(n);
    const double* cb = a.pool + (CN ? in.coef_cn : in.coef_ie);
    const double* et = a.exptab + (CN ? in.exp_cn : in.exp_ie);
    const int steps = CN ? in.Mf : in.Mg;
    __syncthreads();  // the previous task is done with the shared tables
    load_solver<M, NW, C, S2>(cb, sm, rg);
    if constexpr (C > 1) cg::this_cluster().sync();  // every CTA of the grid holds its tables

    const int Nx = in.Nx;
    const int g = c * T + t;
    double num = 0.0, den = 0.0;
    if (mine) {
      const double* Vin = a.in + (a.in_state ? in.state_off : in.slice_off) + (int64_t)n * Nx;
      double W[M], x[M];
      load_state<M, NW, C, S2>(in, Vin, sm, rg, W);
#pragma unroll
      for (int k = 0; k < M; ++k) x[k] = 0.0;
      run_slice<M, NW, C, CN, S2>(in, slice_KeN(in, n), et, steps, W, x, sm, rg, seq);

      const bool first_thread = c == 0 && t == 0;
      const bool last_thread = c == C - 1 && t == T - 1;
      const double Bend = bc_right(in, n + 1);
      double* Vout = a.out + (a.out_state ? in.state_off + (int64_t)(n + 1) * Nx : in.slice_off + (int64_t)n * Nx);
      if (a.mode == PropArgs::kPlain) {
#pragma unroll
        for (int k = 0; k < M; ++k) {
          const int j = g * M + k - in.Np + 1;
          if (j >= 1 && j <= Nx - 2) Vout[j] = row_value<M, NW, C, CN>(cb, k, W, x, rg.isigp);
        }
        if (first_thread) Vout[0] = 0.0;
        if (last_thread) Vout[Nx - 1] = Bend;
      } else {
        // kPinnFused: U^{k+1}_{n+1} = F(U^k_n) + (G_new - G_old) with G = the network
        // table at tau_{n+1} for both terms (Eq. 7), so G_new - G_old = 0 and the
        // update is F itself; increment-norm partial sums.  A non-finite table
        // value needs no check here: it is in U^0 (the initial iterate), so the
        // first iteration's increment norm is not finite and the solve stops
        // with BS_DIVERGED.
        const double* Uold = a.uold + in.state_off + (int64_t)(n + 1) * Nx;
#pragma unroll
        for (int k = 0; k < M; ++k) {
          const int j = g * M + k - in.Np + 1;
          if (j >= 1 && j <= Nx - 2) {
            const double v = row_value<M, NW, C, CN>(cb, k, W, x, rg.isigp);
            Vout[j] = v;
            const double d = v - Uold[j];
            num = fma(d, d, num);
            den = fma(v, v, den);
          }
        }
        if (first_thread) {
          const double v = 0.0;
          Vout[0] = v;
          const double d = v - Uold[0];
          num = fma(d, d, num);
          den = fma(v, v, den);
        }
        if (last_thread) {
          const double v = Bend;
          Vout[Nx - 1] = v;
          const double d = v - Uold[Nx - 1];
          num = fma(d, d, num);
          den = fma(v, v, den);
        }
        // the slice that becomes exact this iteration keeps its start value
        if (a.k_iter >= 0 && n == a.k_iter) {
          double* Fz = a.out + in.state_off + (int64_t)n * Nx;
          for (int j = g; j < Nx; j += C * T) Fz[j] = Vin[j];
        }
      }
    }
    if (a.mode == PropArgs::kPinnFused) {
      block_sum2<NW>(num, den, sm.red[gi]);  // every thread of the CTA
      if (mine && t == 0) {
        const int64_t slot = (in.norm_off + (int64_t)(n + 1) * C + c) * 2;
        a.normbuf[slot + 0] = num;
        a.normbuf[slot + 1] = den;
      }
    }
    if constexpr (C > 1) cg::this_cluster().sync();  // no CTA moves on while its tables may be read
  }
  exchange_drain<M, NW, C, S2>(sm, rg, seq, a.status);
  if constexpr (C > 1) cg::this_cluster().sync();  // no CTA leaves while its shared memory may be written
}

// Classical serial fine time stepping (Eq. 6): one cluster per instance walks
// the slices; every slice restarts from the stored vector, exactly like an
// independent fine_propagate call on that slice.
template <int M, int NW, int C>
__global__ void __launch_bounds__(NW * 32, 1) serial_fine_kernel(SerialArgs a) {
  constexpr int T = NW * 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SolverSmem<M, NW, C>& sm = *reinterpret_cast<SolverSmem<M, NW, C>*>(smem_raw);
  const Inst in = a.insts[a.ids[blockIdx.y]];
  const int t = threadIdx.x, Nx = in.Nx, c = cta_rank<C>();
  const int g = c * T + t;
  const double* cb = a.pool + in.coef_cn;
  const double* et = a.exptab + in.exp_cn;
  SolverRegs rg;
  exchange_init<M, NW, C>(sm, rg);
  load_solver<M, NW, C>(cb, sm, rg);
  double* U = a.out + in.state_off;
  for (int j = g; j < Nx; j += C * T) {
    const double S = j * in.dS;
    U[j] = S - in.K > 0.0 ? S - in.K : 0.0;
  }
  if constexpr (C > 1) {
    cg::this_cluster().sync();
  } else {
    __syncthreads();
  }
  int seq = 0;
  for (int n = 0; n < in.P; ++n) {
    double W[M], x[M];
    load_state<M, NW, C>(in, U + (int64_t)n * Nx, sm, rg, W);
#pragma unroll
    for (int k = 0; k < M; ++k) x[k] = 0.0;
    run_slice<M, NW, C, true>(in, in.K * __ldg(a.exptab + in.exp_sl + n), et, in.Mf, W, x, sm, rg, seq);
    double* Vout = U + (int64_t)(n + 1) * Nx;
#pragma unroll
    for (int k = 0; k < M; ++k) {
      const int j = g * M + k - in.Np + 1;
      if (j >= 1 && j <= Nx - 2) Vout[j] = row_value<M, NW, C, true>(cb, k, W, x, rg.isigp);
    }
    if (c == 0 && t == 0) Vout[0] = 0.0;
    if (c == C - 1 && t == T - 1) Vout[Nx - 1] = bc_right(in, a.exptab + in.exp_sl, n + 1);
    // the next slice reads values other CTAs wrote (global memory, cluster scope)
    __threadfence();
    if constexpr (C > 1) {
      cg::this_cluster().sync();
    } else {
      __syncthreads();
    }
  }
  exchange_drain<M, NW, C>(sm, rg, seq, a.status);
  if constexpr (C > 1) cg::this_cluster().sync();
}

// ---------------------------------------------------------------------------
// Serial coarse sweep with the Parareal correction (Eq. 7), one cluster per
// instance.  IE: G = coarse_steps implicit Euler steps.  Increment kind:
// G(V) = V + g_{n+1} - g_n (elementwise).  Network-anchored IE: G(V) = IE(V) +
// c_n at the interior nodes, c_n = g_{n+1} - IE(g_n) stored in slot n+1 of the
// table (table_correction_kernel).  k_iter < 0 is the initial sweep
// U^0_{n+1} = G(U^0_n).
// ---------------------------------------------------------------------------
template <int M, int NW, int C>
__global__ void __launch_bounds__(NW * 32, 1) sweep_kernel(SweepArgs a) {
  constexpr int T = NW * 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SolverSmem<M, NW, C, 1, true>& sm = *reinterpret_cast<SolverSmem<M, NW, C, 1, true>*>(smem_raw);
  if (a.n_live != nullptr && *a.n_live == 0) return;  // every instance has converged
  const int idx = a.ids[blockIdx.y];
  const Inst in = a.insts[idx];
  if (a.ctrl != nullptr && a.ctrl[idx].done) return;  // uniform over the cluster
  const int t = threadIdx.x, Nx = in.Nx, c = cta_rank<C>();
  const int g = c * T + t;
  const bool first_thread = c == 0 && t == 0;
  const bool last_thread = c == C - 1 && t == T - 1;
  const bool ie = a.kind != 1;     // kinds 0 and 2 take implicit Euler steps
  const bool anchored = a.kind == 2;
  const double* cb = a.pool + in.coef_ie;
  const double* et = a.exptab + in.exp_ie;
  SolverRegs rg{};
  exchange_init<M, NW, C>(sm, rg);
  if (ie) load_solver<M, NW, C>(cb, sm, rg);
  if constexpr (C > 1) cg::this_cluster().sync();
  const bool init = a.k_iter < 0;
  const int n0 = init ? 0 : a.k_iter;
  // five distinct buffers: no store below can change a value loaded from another
  double* __restrict__ Un = a.unext + in.state_off;          // U^{k+1}
  const double* __restrict__ Uc = a.ucur + in.state_off;     // U^k
  double* __restrict__ Gold = a.gold + in.slice_off;         // G(U^k_n), P slices
  const double* __restrict__ Fv = a.fbuf + in.slice_off;     // F(U^k_n), P slices
  const double* __restrict__ gt = a.gtab + in.state_off;     // network table
  // iteration k starts from U^{k+1}_k = U^k_k (exact since iteration k-1);
  // the initial sweep starts from the payoff already in slot 0
  const double* Vs = (init ? Un : Uc) + (int64_t)n0 * Nx;
  double V[M];
#pragma unroll
  for (int k = 0; k < M; ++k) {
    const int j = g * M + k - in.Np + 1;
    V[k] = (j >= 1 && j <= Nx - 2) ? Vs[j] : 0.0;
  }
  double V0 = Vs[0], VB = Vs[Nx - 1];
  if (!init) {
    for (int j = g; j < Nx; j += C * T) Un[(int64_t)n0 * Nx + j] = Vs[j];
  }
  int seq = 0;
  // few rows per thread: the rows' 1/sigma (constant over the slices) once, and
  // each slice's F, old G and U^k before its step, so that no global load waits
  // behind the step (more rows would not fit in registers)
  constexpr bool kAhead = M <= 4;
  double irow[kAhead ? M : 1];
  if constexpr (kAhead) {
#pragma unroll
    for (int k = 0; k < M; ++k) irow[k] = (k < M - 1) ? cb[coef_rows_off(5, k, g, M, C * T)] : rg.isigp;
  }
  for (int n = n0; n < in.P; ++n) {
    double Gv[M];
    double G0, GB;
    double fa[kAhead ? M : 1], ga[kAhead ? M : 1], oa[kAhead ? M : 1], ca[kAhead ? M : 1];
    if constexpr (!kAhead) {
      // this slice's F, old G, U^k and table rows of the thread into L2 while the
      // coarse step runs (its M rows span at most two 128-byte lines per array)
      const int ja = max(g * M - in.Np + 1, 0), jb = min(g * M + M - in.Np, Nx - 1);
      if (ja <= jb) {
        if (!init) {
          prefetch_l2(Fv + (int64_t)n * Nx + ja);
          prefetch_l2(Fv + (int64_t)n * Nx + jb);
          prefetch_l2(Gold + (int64_t)n * Nx + ja);
          prefetch_l2(Gold + (int64_t)n * Nx + jb);
          prefetch_l2(Uc + (int64_t)(n + 1) * Nx + ja);
          prefetch_l2(Uc + (int64_t)(n + 1) * Nx + jb);
        }
        if (anchored) {
          prefetch_l2(gt + (int64_t)(n + 1) * Nx + ja);
          prefetch_l2(gt + (int64_t)(n + 1) * Nx + jb);
        }
      }
    }
    if constexpr (kAhead) {
#pragma unroll
      for (int k = 0; k < M; ++k) {
        const int j = g * M + k - in.Np + 1;
        const bool in_row = j >= 1 && j <= Nx - 2;
        fa[k] = (in_row && !init) ? Fv[(int64_t)n * Nx + j] : 0.0;
        ga[k] = (in_row && !init) ? Gold[(int64_t)n * Nx + j] : 0.0;
        oa[k] = (in_row && !init) ? Uc[(int64_t)(n + 1) * Nx + j] : 0.0;
        ca[k] = (in_row && anchored) ? gt[(int64_t)(n + 1) * Nx + j] : 0.0;
      }
    }
    if (ie) {
      double W[M], x[M];
#pragma unroll
      for (int k = 0; k < M; ++k) {
        const int j = g * M + k - in.Np + 1;
        const double v = (j >= 1 && j <= Nx - 2) ? V[k] : 0.0;
        W[k] = (k < M - 1) ? sm.rows[2][k][t] * v : rg.sigp * v;
        x[k] = 0.0;
      }
      run_slice<M, NW, C, false>(in, in.K * __ldg(a.exptab + in.exp_sl + n), et, in.Mg, W, x, sm, rg, seq);
#pragma unroll
      for (int k = 0; k < M; ++k) {
        if constexpr (kAhead) {
          Gv[k] = W[k] * irow[k];
        } else {
          Gv[k] = row_value<M, NW, C, false>(cb, k, W, x, rg.isigp);
        }
      }
      if (anchored) {  // + c_n at the interior nodes; Dirichlet nodes stay IE's exact values
#pragma unroll
        for (int k = 0; k < M; ++k) {
          const int j = g * M + k - in.Np + 1;
          if (j >= 1 && j <= Nx - 2) Gv[k] = Gv[k] + (kAhead ? ca[k] : gt[(int64_t)(n + 1) * Nx + j]);
        }
      }
      G0 = 0.0;
      GB = bc_right(in, a.exptab + in.exp_sl, n + 1);
    } else {
#pragma unroll
      for (int k = 0; k < M; ++k) {
        const int j = g * M + k - in.Np + 1;
        Gv[k] = (j >= 1 && j <= Nx - 2) ? V[k] + (gt[(int64_t)(n + 1) * Nx + j] - gt[(int64_t)n * Nx + j]) : 0.0;
      }
      G0 = V0 + (gt[(int64_t)(n + 1) * Nx] - gt[(int64_t)n * Nx]);
      GB = VB + (gt[(int64_t)(n + 1) * Nx + Nx - 1] - gt[(int64_t)n * Nx + Nx - 1]);
    }
    double num = 0.0, den = 0.0;
    double* __restrict__ out = Un + (int64_t)(n + 1) * Nx;
    const double* __restrict__ old = Uc + (int64_t)(n + 1) * Nx;
    double* __restrict__ go = Gold + (int64_t)n * Nx;
    const double* __restrict__ fv = Fv + (int64_t)n * Nx;
    // rows in chunks of KC: all loads of a chunk before its stores, so that a
    // chunk costs one memory round trip (4 rows at M = 32, where registers run out)
    constexpr int KC = kAhead ? M : (M < 8 ? M : (M >= 32 ? 4 : 8));
#pragma unroll
    for (int k0 = 0; k0 < M; k0 += KC) {
      double fj[KC], gj[KC], oj[KC];
#pragma unroll
      for (int q = 0; q < KC; ++q) {
        const int k = k0 + q;
        const int j = g * M + k - in.Np + 1;
        const bool in_row = j >= 1 && j <= Nx - 2 && !init;
        fj[q] = kAhead ? fa[k] : (in_row ? fv[j] : 0.0);
        gj[q] = kAhead ? ga[k] : (in_row ? go[j] : 0.0);
        oj[q] = kAhead ? oa[k] : (in_row ? old[j] : 0.0);
      }
#pragma unroll
      for (int q = 0; q < KC; ++q) {
        const int k = k0 + q;
        const int j = g * M + k - in.Np + 1;
        if (j >= 1 && j <= Nx - 2) {
          const double v = init ? Gv[k] : fj[q] + (Gv[k] - gj[q]);
          go[j] = Gv[k];
          out[j] = v;
          V[k] = v;
          if (!init) {
            const double d = v - oj[q];
            num = fma(d, d, num);
            den = fma(v, v, den);
          }
        }
      }
    }
    // Dirichlet nodes follow the same formula (exact values in, exact out);
    // each is read and written by one thread only
    if (first_thread) {
      const double v0 = init ? G0 : fv[0] + (G0 - go[0]);
      go[0] = G0;
      out[0] = v0;
      V0 = v0;
      if (!init) {
        const double d = v0 - old[0];
        num = fma(d, d, num);
        den = fma(v0, v0, den);
      }
    }
    if (last_thread) {
      const double vB = init ? GB : fv[Nx - 1] + (GB - go[Nx - 1]);
      go[Nx - 1] = GB;
      out[Nx - 1] = vB;
      VB = vB;
      if (!init) {
        const double d = vB - old[Nx - 1];
        num = fma(d, d, num);
        den = fma(vB, vB, den);
      }
    }
    if (!init) {
      block_sum2<NW>(num, den, sm.red[0]);
      if (t == 0) {
        const int64_t slot = (in.norm_off + (int64_t)(n + 1) * C + c) * 2;
        a.normbuf[slot + 0] = num;
        a.normbuf[slot + 1] = den;
      }
    }
    __syncthreads();
  }
  exchange_drain<M, NW, C>(sm, rg, seq, a.status);
  if constexpr (C > 1) cg::this_cluster().sync();
}

// ---------------------------------------------------------------------------
// Small Parareal control kernels.
// ---------------------------------------------------------------------------

// U^0: payoff at slice 0 of both buffers; network table at slices 1..P for the
// state-independent network coarse propagator (U^0_{n+1} = G(U^0_n) = g_{n+1}).
__global__ void parareal_init_kernel(const Inst* insts, int n_inst, double* buf0, double* buf1, const double* gtab,
                                     int pinn, Ctrl* ctrl, double* norms, int max_iter) {
  const int idx = blockIdx.x;
  if (idx >= n_inst) return;
  const Inst in = insts[idx];
  const int Nx = in.Nx;
  for (int j = threadIdx.x; j < Nx; j += blockDim.x) {
    const double S = j * in.dS;
    const double v = S - in.K > 0.0 ? S - in.K : 0.0;
    buf0[in.state_off + j] = v;
    buf1[in.state_off + j] = v;
  }
  if (pinn) {
    for (int64_t i = threadIdx.x; i < (int64_t)in.P * Nx; i += blockDim.x)
      buf0[in.state_off + Nx + i] = gtab[in.state_off + Nx + i];
  }
  for (int i = threadIdx.x; i < max_iter; i += blockDim.x) norms[(int64_t)idx * max_iter + i] = nan("");
  if (threadIdx.x == 0) {
    ctrl[idx].done = 0;
    ctrl[idx].iterations = 0;
    ctrl[idx].status = 4;  // BS_NOT_CONVERGED until proven otherwise
    ctrl[idx].last_norm = nan("");
  }
}

// e_k = max_n ||U^{k+1}_n - U^k_n|| / ||U^{k+1}_n|| over the slices updated in
// iteration k, then the stop rule of parareal_solve.  One warp per instance.
__global__ void parareal_finalize_kernel(const Inst* insts, int n_inst, const double* normbuf, int k, double tol,
                                         int max_iter, Ctrl* ctrl, double* norms, int* live_out) {
  const int idx = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int L = threadIdx.x & 31;
  if (idx >= n_inst) return;
  if (ctrl[idx].done) return;  // uniform over the warp
  const Inst in = insts[idx];
  double e = 0.0;
  bool bad = false;
  for (int i = k + 1 + L; i <= in.P; i += 32) {
    double sn = 0.0, sd = 0.0;
    for (int c = 0; c < in.C; ++c) {
      const int64_t slot = (in.norm_off + (int64_t)i * in.C + c) * 2;
      sn += normbuf[slot];
      sd += normbuf[slot + 1];
    }
    const double num = sqrt(sn), den = sqrt(sd);
    const double q = den > 0.0 ? num / den : num;
    if (!(q == q) || isinf(q)) bad = true;
    if (q > e) e = q;
  }
  for (int s = 16; s >= 1; s >>= 1) {
    const double o = __shfl_xor_sync(kFull, e, s);
    e = o > e ? o : e;
  }
  bad = __any_sync(kFull, bad);
  if (L != 0) return;
  norms[(int64_t)idx * max_iter + k] = bad ? nan("") : e;
  ctrl[idx].iterations = k + 1;
  ctrl[idx].last_norm = bad ? nan("") : e;
  if (bad) {
    ctrl[idx].done = 1;
    ctrl[idx].status = 5;  // BS_DIVERGED
  } else if (e <= tol || k + 1 >= in.P) {
    ctrl[idx].done = 1;
    ctrl[idx].status = 0;
  } else if (k + 1 >= max_iter) {
    ctrl[idx].done = 1;
    ctrl[idx].status = 4;
  } else if (live_out != nullptr) {
    atomicAdd(live_out, 1);  // still iterating after iteration k
  }
}

__global__ void parareal_copy_result_kernel(const Inst* insts, int n_inst, const Ctrl* ctrl, const double* buf0,
                                            const double* buf1, double* out) {
  const int idx = blockIdx.y;
  if (idx >= n_inst) return;
  const Inst in = insts[idx];
  const double* src = (ctrl[idx].iterations & 1) ? buf1 : buf0;
  const int64_t sz = (int64_t)(in.P + 1) * in.Nx;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < sz; i += (int64_t)gridDim.x * blockDim.x)
    out[in.state_off + i] = src[in.state_off + i];
}

// Grid points (S_j, tau_n) [, sigma, r, K] of every instance for the network table.
__global__ void grid_points_kernel(const Inst* insts, int n_inst, int d_in, double* X) {
  const int idx = blockIdx.y;
  if (idx >= n_inst) return;
  const Inst in = insts[idx];
  const int64_t sz = (int64_t)(in.P + 1) * in.Nx;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < sz; i += (int64_t)gridDim.x * blockDim.x) {
    const int n = (int)(i / in.Nx), j = (int)(i % in.Nx);
    double* x = X + (in.state_off + i) * d_in;
    x[0] = j * in.dS;
    x[1] = in.T * (double)n / (double)in.P;
    if (d_in >= 5) {
      x[2] = in.sigma;
      x[3] = in.r;
      x[4] = in.K;
    }
  }
}

// Dirichlet nodes of the network table replaced by the exact values.
__global__ void table_fix_kernel(const Inst* insts, int n_inst, const double* exptab, double* g) {
  const int idx = blockIdx.x;
  if (idx >= n_inst) return;
  const Inst in = insts[idx];
  for (int n = threadIdx.x; n <= in.P; n += blockDim.x) {
    g[in.state_off + (int64_t)n * in.Nx] = 0.0;
    g[in.state_off + (int64_t)n * in.Nx + in.Nx - 1] = bc_right(in, exptab + in.exp_sl, n);
  }
}

// Network-anchored IE coarse propagator: slot n+1 of the table becomes the
// correction c_n = g_{n+1} - IE(g_n) at the interior nodes (0 at the Dirichlet
// nodes); gie holds IE(g_n) for n = 0..P-1 in slice layout.  Slot 0 keeps g_0.
__global__ void table_correction_kernel(const Inst* insts, int n_inst, const double* gie, double* g) {
  const int idx = blockIdx.y;
  if (idx >= n_inst) return;
  const Inst in = insts[idx];
  const int64_t sz = (int64_t)in.P * in.Nx;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < sz; i += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(i % in.Nx);
    double* c = g + in.state_off + in.Nx + i;
    *c = (j == 0 || j == in.Nx - 1) ? 0.0 : *c - gie[in.slice_off + i];
  }
}

// ---------------------------------------------------------------------------
// Host-side dispatch over the (M, NW, C) partition classes.
// ---------------------------------------------------------------------------

#define BSP_FOR_EACH_CLASS(X)                                                                        \
  X(2, 1, 1) X(4, 1, 1) X(8, 1, 1) X(16, 1, 1) X(32, 1, 1) X(2, 2, 1) X(4, 2, 1) X(8, 2, 1) X(16, 2, 1) \
  X(32, 2, 1) X(2, 4, 1) X(4, 4, 1) X(8, 4, 1) X(16, 4, 1) X(32, 4, 1) X(2, 4, 2) X(4, 4, 2)             \
  X(8, 4, 2) X(16, 4, 2) X(32, 4, 2) X(2, 4, 4) X(4, 4, 4) X(8, 4, 4) X(16, 4, 4) X(32, 4, 4)         \
  X(2, 4, 8) X(4, 4, 8) X(8, 4, 8) X(16, 4, 8) X(32, 4, 8) X(4, 4, 16) X(8, 4, 16) X(16, 4, 16)       \
  X(32, 4, 16) X(32, 8, 8)

bool partition_supported(int M, int NW, int C) {
#define X(MM, WW, CC) \
  if (M == MM && NW == WW && C == CC) return true;
  BSP_FOR_EACH_CLASS(X)
#undef X
  return false;
}

cudaError_t launch_setup(const Inst* d_insts, const int32_t* d_ids, int n, int Ws, double* pool, double* exptab,
                         cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  setup_rows_kernel<<<dim3(Ws, n), 32, 0, s>>>(d_insts, d_ids, pool, exptab);
  setup_iface_kernel<<<dim3(Ws, n), 32, 0, s>>>(d_insts, d_ids, pool);
  const int smem = (int)(sizeof(double) * (size_t)Ws * (2 * Ws + 1));
  cudaError_t e = cudaFuncSetAttribute(setup_cross_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  setup_cross_kernel<<<dim3(n, 2), 128, smem, s>>>(d_insts, d_ids, pool);
  return cudaGetLastError();
}

template <typename Kern, typename Arg>
static cudaError_t launch_cluster(Kern kernel, dim3 grid, int threads, int C, int smem, cudaStream_t s,
                                  const Arg& arg) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  if (C > 8) {
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, arg);
}

// Persistent launch: as many clusters as fit on the device at once (or one per
// task when there are fewer tasks), each walking its share of the tasks.
template <typename Kern>
static cudaError_t launch_persistent(Kern kernel, int threads, int C, int smem, cudaStream_t s, PropArgs a,
                                     int n_inst, int maxP, int s2) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  if (C > 8 && (e = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) != cudaSuccess)
    return e;
  const int kb = a.k_iter > 0 ? a.k_iter : 0;
  const int64_t ntask = maxP > kb ? (int64_t)n_inst * ((maxP - kb + s2 - 1) / s2) : 0;
  if (ntask <= 0) return cudaSuccess;  // no slice from kb on
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3((unsigned)(ntask < 65536 ? ntask : 65536) * C, 1, 1);
  int resident = 0;
  if ((e = cudaOccupancyMaxActiveClusters(&resident, kernel, &cfg)) != cudaSuccess) return e;
  if (resident < 1) resident = 1;
  const int64_t ncl = ntask < resident ? ntask : resident;
  cfg.gridDim = dim3((unsigned)(ncl * C), 1, 1);
  a.n_inst = n_inst;
  a.maxP = maxP;
  return cudaLaunchKernelEx(&cfg, kernel, a);
}

// Classes whose fine propagation can also run two slices per CTA (16 or more
// rows per thread: the tables are large, and two slices of one instance share
// one copy; one-CTA grids step on a named barrier per slice, clusters on their
// mbarriers).
#define BSP_FOR_EACH_S2_CLASS(X)                                                                  \
  X(16, 2, 1) X(32, 1, 1) X(32, 2, 1) X(16, 4, 1) X(32, 4, 1) X(16, 4, 2) X(32, 4, 2) X(16, 4, 4)      \
  X(32, 4, 4) X(16, 4, 8) X(32, 4, 8) X(16, 4, 16) X(32, 4, 16)

bool s2_supported(int M, int NW, int C) {
#define X(MM, WW, CC) \
  if (M == MM && NW == WW && C == CC) return true;
  BSP_FOR_EACH_S2_CLASS(X)
#undef X
  return false;
}

cudaError_t launch_prop(int M, int NW, int C, int s2, bool cn, const PropArgs& a, int n_inst, int maxP,
                        cudaStream_t s) {
  if (n_inst <= 0) return cudaSuccess;
  if (s2 == 2 && cn) {
#define X(MM, WW, CC)                                                                                          \
  if (M == MM && NW == WW && C == CC) {                                                                        \
    const int sz = (int)sizeof(SolverSmem<MM, WW, CC, 2>);                                                     \
    return launch_persistent(prop_kernel<MM, WW, CC, true, 2>, 2 * WW * 32, CC, sz, s, a, n_inst, maxP, 2);    \
  }
    BSP_FOR_EACH_S2_CLASS(X)
#undef X
    return cudaErrorInvalidValue;
  }
#define X(MM, WW, CC)                                                                                            \
  if (M == MM && NW == WW && C == CC) {                                                                          \
    const int sz = (int)sizeof(SolverSmem<MM, WW, CC>), sz_ie = (int)sizeof(SolverSmem<MM, WW, CC, 1, true>);    \
    return cn ? launch_persistent(prop_kernel<MM, WW, CC, true, 1>, WW * 32, CC, sz, s, a, n_inst, maxP, 1)      \
              : launch_persistent(prop_kernel<MM, WW, CC, false, 1>, WW * 32, CC, sz_ie, s, a, n_inst, maxP, 1);  \
  }
  BSP_FOR_EACH_CLASS(X)
#undef X
  return cudaErrorInvalidValue;
}

cudaError_t launch_serial(int M, int NW, int C, const SerialArgs& a, int n_inst, cudaStream_t s) {
  if (n_inst <= 0) return cudaSuccess;
  dim3 grid(C, n_inst);
#define X(MM, WW, CC)                                                                             \
  if (M == MM && NW == WW && C == CC) {                                                           \
    const int sz = (int)sizeof(SolverSmem<MM, WW, CC>);                                           \
    return launch_cluster(serial_fine_kernel<MM, WW, CC>, grid, WW * 32, CC, sz, s, a);           \
  }
  BSP_FOR_EACH_CLASS(X)
#undef X
  return cudaErrorInvalidValue;
}

cudaError_t launch_sweep(int M, int NW, int C, const SweepArgs& a, int n_inst, cudaStream_t s) {
  if (n_inst <= 0) return cudaSuccess;
  dim3 grid(C, n_inst);
#define X(MM, WW, CC)                                                                        \
  if (M == MM && NW == WW && C == CC) {                                                      \
    const int sz = (int)sizeof(SolverSmem<MM, WW, CC, 1, true>);                             \
    return launch_cluster(sweep_kernel<MM, WW, CC>, grid, WW * 32, CC, sz, s, a);            \
  }
  BSP_FOR_EACH_CLASS(X)
#undef X
  return cudaErrorInvalidValue;
}

cudaError_t launch_parareal_init(const Inst* d_insts, int n_inst, double* buf0, double* buf1, const double* gtab,
                                 int pinn, Ctrl* ctrl, double* norms, int max_iter, cudaStream_t s) {
  parareal_init_kernel<<<n_inst, 256, 0, s>>>(d_insts, n_inst, buf0, buf1, gtab, pinn, ctrl, norms, max_iter);
  return cudaGetLastError();
}

cudaError_t launch_parareal_finalize(const Inst* d_insts, int n_inst, const double* normbuf, int k, double tol,
                                     int max_iter, Ctrl* ctrl, double* norms, int* live_out, cudaStream_t s) {
  parareal_finalize_kernel<<<(n_inst + 3) / 4, 128, 0, s>>>(d_insts, n_inst, normbuf, k, tol, max_iter, ctrl, norms,
                                                            live_out);
  return cudaGetLastError();
}

cudaError_t launch_copy_result(const Inst* d_insts, int n_inst, const Ctrl* ctrl, const double* buf0,
                               const double* buf1, double* out, cudaStream_t s) {
  parareal_copy_result_kernel<<<dim3(16, n_inst), 256, 0, s>>>(d_insts, n_inst, ctrl, buf0, buf1, out);
  return cudaGetLastError();
}

cudaError_t launch_grid_points(const Inst* d_insts, int n_inst, int d_in, double* X, cudaStream_t s) {
  grid_points_kernel<<<dim3(16, n_inst), 256, 0, s>>>(d_insts, n_inst, d_in, X);
  return cudaGetLastError();
}

cudaError_t launch_table_fix(const Inst* d_insts, int n_inst, const double* exptab, double* g, cudaStream_t s) {
  table_fix_kernel<<<n_inst, 64, 0, s>>>(d_insts, n_inst, exptab, g);
  return cudaGetLastError();
}

cudaError_t launch_table_correction(const Inst* d_insts, int n_inst, const double* gie, double* g, cudaStream_t s) {
  table_correction_kernel<<<dim3(16, n_inst), 256, 0, s>>>(d_insts, n_inst, gie, g);
  return cudaGetLastError();
}

}  // namespace bsp
