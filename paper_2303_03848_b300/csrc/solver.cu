// solver.cu -- Crank-Nicolson fine propagator, implicit Euler coarse
// propagator and the Parareal iteration (Eq. 7) on sm_103a.
//
// Section 3.2 of the paper: centred differences in S (Eq. 10), Crank-Nicolson
// for F and implicit Euler for G, both one tridiagonal solve per step.
//
// FP64 on this part issues one warp-wide DFMA per 64 cycles per SM
// sub-partition with a dependent-issue latency of the same length, so the
// cost of a step is the number of warp-level FP64 instructions it issues.  The
// design keeps that count near 5 per grid row per step:
//   * Crank-Nicolson is rewritten with Z = V^{m+1} + V^m:
//       (I - h L) Z = 2 V^m + boundary,  V^{m+1} = Z - V^m,  h = dtau/2,
//     and the state is carried scaled, W = 2 V / delta (delta = local LU
//     pivots), so the forward sweep needs no separate right-hand side product.
//   * Each thread eliminates its M-1 inner rows with a local Thomas sweep
//     (factorised once at set-up); the M-th row of every thread forms a
//     tridiagonal interface system that one warp solves by parallel cyclic
//     reduction over shuffles (multipliers precomputed); a tiny dense system
//     couples the warps of a CTA.  A final fixup adds the interface responses
//     to the inner rows.
// The whole grid stays in registers and shared memory for all steps of a slice.
#include <cmath>
#include <cstdio>

#include "bs_common.cuh"
#include "bs_internal.h"

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

__global__ void __launch_bounds__(128) setup_kernel(const Inst* insts, const int32_t* ids, double* pool,
                                                    double* exptab) {
  const Inst in = insts[ids[blockIdx.x]];
  const int kind = blockIdx.y;  // 0: Crank-Nicolson (fine), 1: implicit Euler (coarse)
  const int NW = in.NW, M = in.M, T = NW * 32;
  const int t = threadIdx.x;
  const int L = t & 31;
  const int steps = kind == 0 ? in.Mf : in.Mg;
  const double dt = in.T / ((double)in.P * (double)steps);
  const double h = kind == 0 ? 0.5 * dt : dt;
  const double crhs = kind == 0 ? 2.0 : 1.0;
  double* cb = pool + (kind == 0 ? in.coef_cn : in.coef_ie);
  double* et = exptab + (kind == 0 ? in.exp_cn : in.exp_ie);

  __shared__ double s_alp0[128], s_bet0[128], s_A[128], s_C[128], s_ra[128], s_rc[128];

  for (int m = t; m <= steps; m += blockDim.x) et[m] = exp(-in.r * ((double)m * dt));

  const bool act = t < T;
  double alp_last = 0.0, bet_last = 0.0;
  if (act) {
    // local LU of the M-1 inner rows of thread t
    double lam[32], mu[32], del[32];
    double prev_u = 0.0;
    for (int k = 0; k < M - 1; ++k) {
      const int r = t * M + k;
      double l, d, u;
      mat_row(in, h, r, l, d, u);
      del[k] = (k == 0) ? d : d - l * (prev_u / del[k - 1]);
      lam[k] = l / del[k];
      mu[k] = u / del[k];
      prev_u = u;
      const bool pad = r < in.Np;
      cb[coef_rows_off(0, k, t, M, T)] = lam[k];
      cb[coef_rows_off(1, k, t, M, T)] = mu[k];
      cb[coef_rows_off(2, k, t, M, T)] = pad ? 0.0 : crhs / del[k];
      cb[coef_rows_off(5, k, t, M, T)] = pad ? 0.0 : del[k] / crhs;
    }
    // responses of the inner rows to the left interface X_{t-1} (alpha) and
    // the right interface X_t (beta)
    double phi[32];
    phi[0] = -lam[0];
    for (int k = 1; k < M - 1; ++k) phi[k] = -lam[k] * phi[k - 1];
    double alp = phi[M - 2], bet = -mu[M - 2];
    cb[coef_rows_off(3, M - 2, t, M, T)] = alp;
    cb[coef_rows_off(4, M - 2, t, M, T)] = bet;
    alp_last = alp;
    bet_last = bet;
    for (int k = M - 3; k >= 0; --k) {
      alp = phi[k] - mu[k] * alp;
      bet = -mu[k] * bet;
      cb[coef_rows_off(3, k, t, M, T)] = alp;
      cb[coef_rows_off(4, k, t, M, T)] = bet;
    }
    for (int q = 0; q < 6; ++q) cb[coef_rows_off(q, M - 1, t, M, T)] = 0.0;  // interface row slots unused
    s_alp0[t] = alp;
    s_bet0[t] = bet;
  }
  __syncthreads();
  if (act) {
    double A = 0.0, C = 0.0, kap = 0.0, nu = 0.0, sigp = 0.0, isigp = 0.0;
    if (t < T - 1) {
      // interface row p: l x_{p-1} + d x_p + u x_{p+1} = r_p with the inner
      // neighbours written through their interface responses, divided by D
      const int p = t * M + M - 1;
      double l, d, u;
      mat_row(in, h, p, l, d, u);
      const double D = d + l * bet_last + u * s_alp0[t + 1];
      A = l * alp_last / D;
      C = u * s_bet0[t + 1] / D;
      kap = l / D;
      nu = u / D;
      const bool pad = p < in.Np;
      sigp = pad ? 0.0 : crhs / D;
      isigp = pad ? 0.0 : D / crhs;
    }
    cb[coef_if_off(0, t, M, T)] = kap;
    cb[coef_if_off(1, t, M, T)] = nu;
    cb[coef_if_off(2, t, M, T)] = sigp;
    cb[coef_if_off(3, t, M, T)] = isigp;
    cb[coef_if_off(4, t, M, T)] = A;
    cb[coef_if_off(5, t, M, T)] = C;

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
      cb[coef_pcr_off(lv, t, M, T)] = k1;
      cb[coef_pcr_off(5 + lv, t, M, T)] = k2;
    }
    const double inv = 1.0 / d_;
    cb[coef_pcr_off(10, t, M, T)] = inv;
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
    const double ra = (L == 31) ? 0.0 : ea * inv;
    const double rc = (L == 31) ? 0.0 : ec * inv;
    cb[coef_resp_off(0, t, M, T)] = ra;
    cb[coef_resp_off(1, t, M, T)] = rc;
    s_A[t] = A;
    s_C[t] = C;
    s_ra[t] = ra;
    s_rc[t] = rc;
  }
  __syncthreads();
  if (t == 0) {
    // cross-warp system over Y_w = X at lane 31 of warp w; Y_{NW-1} is the Dirichlet row
    double Mx[kMaxNW][2 * kMaxNW];
    for (int i = 0; i < NW; ++i)
      for (int j = 0; j < 2 * NW; ++j) Mx[i][j] = (j == NW + i) ? 1.0 : 0.0;
    for (int w = 0; w < NW; ++w) {
      if (w == NW - 1) {
        Mx[w][w] = 1.0;
        continue;
      }
      const int t31 = 32 * w + 31, t30 = 32 * w + 30, tn0 = 32 * (w + 1);
      const double A31 = s_A[t31], C31 = s_C[t31];
      if (w > 0) Mx[w][w - 1] = A31 * s_ra[t30];
      Mx[w][w] = 1.0 + A31 * s_rc[t30] + C31 * s_ra[tn0];
      Mx[w][w + 1] = C31 * s_rc[tn0];
    }
    // Gauss-Jordan with partial pivoting
    for (int c = 0; c < NW; ++c) {
      int piv = c;
      for (int i = c + 1; i < NW; ++i)
        if (fabs(Mx[i][c]) > fabs(Mx[piv][c])) piv = i;
      if (piv != c)
        for (int j = 0; j < 2 * NW; ++j) {
          const double tmp = Mx[c][j];
          Mx[c][j] = Mx[piv][j];
          Mx[piv][j] = tmp;
        }
      const double ip = 1.0 / Mx[c][c];
      for (int j = 0; j < 2 * NW; ++j) Mx[c][j] *= ip;
      for (int i = 0; i < NW; ++i) {
        if (i == c) continue;
        const double f = Mx[i][c];
        for (int j = 0; j < 2 * NW; ++j) Mx[i][j] -= f * Mx[c][j];
      }
    }
    for (int v = 0; v < NW; ++v)
      for (int u = 0; u < NW; ++u) cb[coef_G_off(v, u, M, T, NW)] = Mx[v][NW + u];
  }
}

// ---------------------------------------------------------------------------
// One time step of the partitioned solver.
// ---------------------------------------------------------------------------

template <int M, int NW>
struct SolverSmem {
  double rows[5][M][NW * 32];  // lambda, mu, sigma, alpha, beta
  double A31[NW], C31[NW], G[NW * NW];
  double x0[NW], X0[NW], X30[NW], R31[NW];
  double red[2][NW];
};

struct SolverRegs {
  double kap, nu, sigp, isigp;
  double m1[kPcrLevels], m2[kPcrLevels], inv, ra, rc;
};

template <int M, int NW>
__device__ __forceinline__ void load_solver(const double* __restrict__ cb, SolverSmem<M, NW>& sm, SolverRegs& rg) {
  constexpr int T = NW * 32;
  const int t = threadIdx.x;
  double* dst = &sm.rows[0][0][0];
  for (int i = t; i < 5 * M * T; i += T) dst[i] = cb[i];  // rows [q][k][t], q = 0..4, same order
  rg.kap = cb[coef_if_off(0, t, M, T)];
  rg.nu = cb[coef_if_off(1, t, M, T)];
  rg.sigp = cb[coef_if_off(2, t, M, T)];
  rg.isigp = cb[coef_if_off(3, t, M, T)];
#pragma unroll
  for (int lv = 0; lv < kPcrLevels; ++lv) {
    rg.m1[lv] = cb[coef_pcr_off(lv, t, M, T)];
    rg.m2[lv] = cb[coef_pcr_off(5 + lv, t, M, T)];
  }
  rg.inv = cb[coef_pcr_off(10, t, M, T)];
  rg.ra = cb[coef_resp_off(0, t, M, T)];
  rg.rc = cb[coef_resp_off(1, t, M, T)];
  if (t < NW) {
    sm.A31[t] = cb[coef_if_off(4, 32 * t + 31, M, T)];
    sm.C31[t] = cb[coef_if_off(5, 32 * t + 31, M, T)];
  }
  if (t < NW * NW) sm.G[t] = cb[coef_G_off(t / NW, t % NW, M, T, NW)];
  __syncthreads();
}

// x receives the solution of the step (Z for Crank-Nicolson, V^{m+1} for
// implicit Euler) on the thread's rows; W is advanced to the next scaled state.
template <int M, int NW, bool CN>
__device__ __forceinline__ void tri_step(double (&W)[M], double (&x)[M], SolverSmem<M, NW>& sm, const SolverRegs& rg,
                                         double Zb) {
  constexpr int T = NW * 32;
  const int t = threadIdx.x, L = t & 31, w = t >> 5;
  // 1. local forward and backward sweeps over the inner rows (zero interfaces)
  x[0] = W[0];
#pragma unroll
  for (int k = 1; k <= M - 2; ++k) x[k] = fma(-sm.rows[0][k][t], x[k - 1], W[k]);
#pragma unroll
  for (int k = M - 3; k >= 0; --k) x[k] = fma(-sm.rows[1][k][t], x[k + 1], x[k]);
  // 2. interface right-hand side: needs the first inner value of thread t+1
  double xs_next = __shfl_down_sync(kFull, x[0], 1);
  if (L == 0) sm.x0[w] = x[0];
  __syncthreads();
  if (L == 31) xs_next = (w + 1 < NW) ? sm.x0[w + 1] : 0.0;
  double R = fma(-rg.nu, xs_next, fma(-rg.kap, x[M - 2], W[M - 1]));
  if (t == T - 1) R = Zb;  // Dirichlet row at Smax
  // 3. in-warp PCR on lanes 0..30 with zero external couplings
  double Rp = (L == 31) ? 0.0 : R;
#pragma unroll
  for (int lv = 0; lv < kPcrLevels; ++lv) {
    const int s = 1 << lv;
    const double up = __shfl_up_sync(kFull, Rp, s);
    const double dn = __shfl_down_sync(kFull, Rp, s);
    Rp = fma(-rg.m1[lv], up, fma(-rg.m2[lv], dn, Rp));
  }
  const double Xt = Rp * rg.inv;
  if (L == 0) sm.X0[w] = Xt;
  if (L == 30) sm.X30[w] = Xt;
  if (L == 31) sm.R31[w] = R;
  __syncthreads();
  // 4. cross-warp unknowns Y_u (lane 31 of warp u): rho_u by lane u, then
  //    Y_{w-1} (lane 0) and Y_w (lane 1) from the precomputed inverse
  double rho = 0.0;
  if (L < NW) {
    rho = (L == NW - 1) ? sm.R31[L] : fma(-sm.C31[L], sm.X0[L + 1], fma(-sm.A31[L], sm.X30[L], sm.R31[L]));
  }
  const int grow = (L == 0) ? w - 1 : w;
  double y = 0.0;
#pragma unroll
  for (int u = 0; u < NW; ++u) {
    const double ru = __shfl_sync(kFull, rho, u);
    const double gc = (grow >= 0) ? sm.G[grow * NW + u] : 0.0;
    y = fma(gc, ru, y);
  }
  const double Yl = __shfl_sync(kFull, y, 0);
  const double Yr = __shfl_sync(kFull, y, 1);
  const double X = (L == 31) ? Yr : fma(rg.rc, Yr, fma(rg.ra, Yl, Xt));
  double Xprev = __shfl_up_sync(kFull, X, 1);
  if (L == 0) Xprev = Yl;
  // 5. fixup of the inner rows and the scaled state update
#pragma unroll
  for (int k = 0; k <= M - 2; ++k) {
    const double xv = fma(sm.rows[4][k][t], X, fma(sm.rows[3][k][t], Xprev, x[k]));
    x[k] = xv;
    W[k] = CN ? fma(sm.rows[2][k][t], xv, -W[k]) : sm.rows[2][k][t] * xv;
  }
  x[M - 1] = X;
  W[M - 1] = CN ? fma(rg.sigp, X, -W[M - 1]) : rg.sigp * X;
}

// Read the Nx-vector V into the thread's rows and scale it into W.
template <int M, int NW>
__device__ __forceinline__ void load_state(const Inst& in, const double* __restrict__ V, const SolverSmem<M, NW>& sm,
                                           const SolverRegs& rg, double (&W)[M]) {
  const int t = threadIdx.x;
#pragma unroll
  for (int k = 0; k < M; ++k) {
    const int j = t * M + k - in.Np + 1;
    const double v = (j >= 1 && j <= in.Nx - 2) ? V[j] : 0.0;
    W[k] = (k < M - 1) ? sm.rows[2][k][t] * v : rg.sigp * v;
  }
}

// Value of row k of this thread after a slice: V = W / sigma (CN) or x (IE).
template <int M, int NW, bool CN>
__device__ __forceinline__ double row_value(const double* __restrict__ cb, int k, const double (&W)[M],
                                            const double (&x)[M], double isigp) {
  if (!CN) return x[k];
  const double is = (k < M - 1) ? cb[coef_rows_off(5, k, threadIdx.x, M, NW * 32)] : isigp;
  return W[k] * is;
}

// Run `steps` steps of the propagator on slice n starting from scaled state W.
template <int M, int NW, bool CN>
__device__ __forceinline__ void run_slice(const Inst& in, int n, const double* __restrict__ et, int steps,
                                          double (&W)[M], double (&x)[M], SolverSmem<M, NW>& sm,
                                          const SolverRegs& rg) {
  const double tau_n = in.T * (double)n / (double)in.P;
  const double KeN = in.K * exp(-in.r * tau_n);
  double Bold = in.Smax - KeN;  // exp(0) = 1
  const bool last_warp = (threadIdx.x >> 5) == NW - 1;
  for (int m = 0; m < steps; ++m) {
    double Zb = 0.0;
    if (last_warp) {
      const double Bnew = fma(-KeN, __ldg(et + m + 1), in.Smax);
      Zb = CN ? Bold + Bnew : Bnew;
      Bold = Bnew;
    }
    tri_step<M, NW, CN>(W, x, sm, rg, Zb);
  }
}

// Block-wide sum of two doubles, result valid on thread 0.
template <int NW>
__device__ __forceinline__ void block_sum2(double& a, double& b, double (*red)[NW]) {
  const int t = threadIdx.x, L = t & 31, w = t >> 5;
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

// ---------------------------------------------------------------------------
// Propagation over slices: fine (Crank-Nicolson) or coarse (implicit Euler).
// One CTA per (instance, slice).
// ---------------------------------------------------------------------------

template <int M, int NW, bool CN>
__global__ void __launch_bounds__(NW * 32, 1) prop_kernel(PropArgs a) {
  constexpr int T = NW * 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SolverSmem<M, NW>& sm = *reinterpret_cast<SolverSmem<M, NW>*>(smem_raw);
  const int idx = a.ids[blockIdx.y];
  const Inst in = a.insts[idx];
  const int n = blockIdx.x;
  if (n >= in.P) return;
  if (a.k_iter >= 0 && n < a.k_iter) return;
  if (a.ctrl != nullptr && a.ctrl[idx].done) return;
  if (a.active != nullptr && !a.active[in.task_off + n]) return;
  const int t = threadIdx.x;
  const double* cb = a.pool + (CN ? in.coef_cn : in.coef_ie);
  const double* et = a.exptab + (CN ? in.exp_cn : in.exp_ie);
  const int steps = CN ? in.Mf : in.Mg;
  SolverRegs rg;
  load_solver<M, NW>(cb, sm, rg);

  const int Nx = in.Nx;
  const double* Vin = a.in + (a.in_state ? in.state_off : in.slice_off) + (int64_t)n * Nx;
  double W[M], x[M];
  load_state<M, NW>(in, Vin, sm, rg, W);
#pragma unroll
  for (int k = 0; k < M; ++k) x[k] = 0.0;
  run_slice<M, NW, CN>(in, n, et, steps, W, x, sm, rg);

  const double Bend = in.Smax - in.K * exp(-in.r * (in.T * (double)(n + 1) / (double)in.P));
  double* Vout = a.out + (a.out_state ? in.state_off + (int64_t)(n + 1) * Nx : in.slice_off + (int64_t)n * Nx);
  if (a.mode == PropArgs::kPlain) {
#pragma unroll
    for (int k = 0; k < M; ++k) {
      const int j = t * M + k - in.Np + 1;
      if (j >= 1 && j <= Nx - 2) Vout[j] = row_value<M, NW, CN>(cb, k, W, x, rg.isigp);
    }
    if (t == 0) Vout[0] = 0.0;
    if (t == T - 1) Vout[Nx - 1] = Bend;
    return;
  }
  // kPinnFused: U^{k+1}_{n+1} = F(U^k_n) + (G_new - G_old) with G = the network
  // table at tau_{n+1} for both terms (Eq. 7); increment-norm partial sums.
  const double* g = a.gtab + in.state_off + (int64_t)(n + 1) * Nx;
  const double* Uold = a.uold + in.state_off + (int64_t)(n + 1) * Nx;
  double num = 0.0, den = 0.0;
#pragma unroll
  for (int k = 0; k < M; ++k) {
    const int j = t * M + k - in.Np + 1;
    if (j >= 1 && j <= Nx - 2) {
      const double f = row_value<M, NW, CN>(cb, k, W, x, rg.isigp);
      const double v = f + (g[j] - g[j]);
      Vout[j] = v;
      const double d = v - Uold[j];
      num = fma(d, d, num);
      den = fma(v, v, den);
    }
  }
  if (t == 0) {
    const double v = 0.0 + (g[0] - g[0]);
    Vout[0] = v;
    const double d = v - Uold[0];
    num = fma(d, d, num);
    den = fma(v, v, den);
  }
  if (t == T - 1) {
    const double v = Bend + (g[Nx - 1] - g[Nx - 1]);
    Vout[Nx - 1] = v;
    const double d = v - Uold[Nx - 1];
    num = fma(d, d, num);
    den = fma(v, v, den);
  }
  // the slice that becomes exact this iteration keeps its start value
  if (a.k_iter >= 0 && n == a.k_iter) {
    double* Fz = a.out + in.state_off + (int64_t)n * Nx;
    for (int j = t; j < Nx; j += T) Fz[j] = Vin[j];
  }
  block_sum2<NW>(num, den, sm.red);
  if (t == 0) {
    a.normbuf[2 * (in.task1_off + n + 1) + 0] = num;
    a.normbuf[2 * (in.task1_off + n + 1) + 1] = den;
  }
}

// Classical serial fine time stepping (Eq. 6): one CTA per instance walks the
// slices; every slice restarts from the stored vector, exactly like an
// independent fine_propagate call on that slice.
template <int M, int NW>
__global__ void __launch_bounds__(NW * 32, 1) serial_fine_kernel(SerialArgs a) {
  constexpr int T = NW * 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SolverSmem<M, NW>& sm = *reinterpret_cast<SolverSmem<M, NW>*>(smem_raw);
  const Inst in = a.insts[a.ids[blockIdx.x]];
  const int t = threadIdx.x, Nx = in.Nx;
  const double* cb = a.pool + in.coef_cn;
  const double* et = a.exptab + in.exp_cn;
  SolverRegs rg;
  load_solver<M, NW>(cb, sm, rg);
  double* U = a.out + in.state_off;
  for (int j = t; j < Nx; j += T) {
    const double S = j * in.dS;
    U[j] = S - in.K > 0.0 ? S - in.K : 0.0;
  }
  __syncthreads();
  for (int n = 0; n < in.P; ++n) {
    double W[M], x[M];
    load_state<M, NW>(in, U + (int64_t)n * Nx, sm, rg, W);
#pragma unroll
    for (int k = 0; k < M; ++k) x[k] = 0.0;
    run_slice<M, NW, true>(in, n, et, in.Mf, W, x, sm, rg);
    double* Vout = U + (int64_t)(n + 1) * Nx;
#pragma unroll
    for (int k = 0; k < M; ++k) {
      const int j = t * M + k - in.Np + 1;
      if (j >= 1 && j <= Nx - 2) Vout[j] = row_value<M, NW, true>(cb, k, W, x, rg.isigp);
    }
    if (t == 0) Vout[0] = 0.0;
    if (t == T - 1) Vout[Nx - 1] = in.Smax - in.K * exp(-in.r * (in.T * (double)(n + 1) / (double)in.P));
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Serial coarse sweep with the Parareal correction (Eq. 7), one CTA per
// instance.  IE: G = coarse_steps implicit Euler steps.  Increment kind:
// G(V) = V + g_{n+1} - g_n (elementwise).  k_iter < 0 is the initial sweep
// U^0_{n+1} = G(U^0_n).
// ---------------------------------------------------------------------------
template <int M, int NW>
__global__ void __launch_bounds__(NW * 32, 1) sweep_kernel(SweepArgs a) {
  constexpr int T = NW * 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SolverSmem<M, NW>& sm = *reinterpret_cast<SolverSmem<M, NW>*>(smem_raw);
  const int idx = a.ids[blockIdx.x];
  const Inst in = a.insts[idx];
  if (a.ctrl != nullptr && a.ctrl[idx].done) return;
  const int t = threadIdx.x, Nx = in.Nx;
  const bool ie = a.kind == 0;
  const double* cb = a.pool + in.coef_ie;
  const double* et = a.exptab + in.exp_ie;
  SolverRegs rg{};
  if (ie) load_solver<M, NW>(cb, sm, rg);
  const bool init = a.k_iter < 0;
  const int n0 = init ? 0 : a.k_iter;
  double* Un = a.unext + in.state_off;          // U^{k+1}
  const double* Uc = a.ucur + in.state_off;     // U^k
  double* Gold = a.gold + in.slice_off;         // G(U^k_n), P slices
  const double* Fv = a.fbuf + in.slice_off;     // F(U^k_n), P slices
  const double* g = a.gtab + in.state_off;      // network table
  // iteration k starts from U^{k+1}_k = U^k_k (exact since iteration k-1);
  // the initial sweep starts from the payoff already in slot 0
  const double* Vs = (init ? Un : Uc) + (int64_t)n0 * Nx;
  double V[M];
#pragma unroll
  for (int k = 0; k < M; ++k) {
    const int j = t * M + k - in.Np + 1;
    V[k] = (j >= 1 && j <= Nx - 2) ? Vs[j] : 0.0;
  }
  double V0 = Vs[0], VB = Vs[Nx - 1];
  if (!init) {
    for (int j = t; j < Nx; j += T) Un[(int64_t)n0 * Nx + j] = Vs[j];
  }
  for (int n = n0; n < in.P; ++n) {
    double Gv[M];
    double G0, GB;
    if (ie) {
      double W[M], x[M];
#pragma unroll
      for (int k = 0; k < M; ++k) {
        const int j = t * M + k - in.Np + 1;
        const double v = (j >= 1 && j <= Nx - 2) ? V[k] : 0.0;
        W[k] = (k < M - 1) ? sm.rows[2][k][t] * v : rg.sigp * v;
        x[k] = 0.0;
      }
      run_slice<M, NW, false>(in, n, et, in.Mg, W, x, sm, rg);
#pragma unroll
      for (int k = 0; k < M; ++k) Gv[k] = x[k];
      G0 = 0.0;
      GB = in.Smax - in.K * exp(-in.r * (in.T * (double)(n + 1) / (double)in.P));
    } else {
#pragma unroll
      for (int k = 0; k < M; ++k) {
        const int j = t * M + k - in.Np + 1;
        Gv[k] = (j >= 1 && j <= Nx - 2) ? V[k] + (g[(int64_t)(n + 1) * Nx + j] - g[(int64_t)n * Nx + j]) : 0.0;
      }
      G0 = V0 + (g[(int64_t)(n + 1) * Nx] - g[(int64_t)n * Nx]);
      GB = VB + (g[(int64_t)(n + 1) * Nx + Nx - 1] - g[(int64_t)n * Nx + Nx - 1]);
    }
    double num = 0.0, den = 0.0;
    double* out = Un + (int64_t)(n + 1) * Nx;
    const double* old = Uc + (int64_t)(n + 1) * Nx;
    double* go = Gold + (int64_t)n * Nx;
    const double* fv = Fv + (int64_t)n * Nx;
#pragma unroll
    for (int k = 0; k < M; ++k) {
      const int j = t * M + k - in.Np + 1;
      if (j >= 1 && j <= Nx - 2) {
        const double v = init ? Gv[k] : fv[j] + (Gv[k] - go[j]);
        go[j] = Gv[k];
        out[j] = v;
        V[k] = v;
        if (!init) {
          const double d = v - old[j];
          num = fma(d, d, num);
          den = fma(v, v, den);
        }
      }
    }
    // Dirichlet nodes follow the same formula (exact values in, exact out)
    const double v0 = init ? G0 : fv[0] + (G0 - go[0]);
    const double vB = init ? GB : fv[Nx - 1] + (GB - go[Nx - 1]);
    __syncthreads();
    if (t == 0) {
      go[0] = G0;
      out[0] = v0;
      if (!init) {
        const double d = v0 - old[0];
        num = fma(d, d, num);
        den = fma(v0, v0, den);
      }
    }
    if (t == T - 1) {
      go[Nx - 1] = GB;
      out[Nx - 1] = vB;
      if (!init) {
        const double d = vB - old[Nx - 1];
        num = fma(d, d, num);
        den = fma(vB, vB, den);
      }
    }
    V0 = v0;
    VB = vB;
    if (!init) {
      block_sum2<NW>(num, den, sm.red);
      if (t == 0) {
        a.normbuf[2 * (in.task1_off + n + 1) + 0] = num;
        a.normbuf[2 * (in.task1_off + n + 1) + 1] = den;
      }
    }
    __syncthreads();
  }
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
// iteration k, then the stop rule of parareal_solve.
__global__ void parareal_finalize_kernel(const Inst* insts, int n_inst, const double* normbuf, int k, double tol,
                                         int max_iter, Ctrl* ctrl, double* norms) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_inst) return;
  if (ctrl[idx].done) return;
  const Inst in = insts[idx];
  double e = 0.0;
  bool bad = false;
  for (int i = k + 1; i <= in.P; ++i) {
    const double num = sqrt(normbuf[2 * (in.task1_off + i)]);
    const double den = sqrt(normbuf[2 * (in.task1_off + i) + 1]);
    const double q = den > 0.0 ? num / den : num;
    if (!(q == q) || isinf(q)) bad = true;
    if (q > e) e = q;
  }
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
__global__ void table_fix_kernel(const Inst* insts, int n_inst, double* g) {
  const int idx = blockIdx.x;
  if (idx >= n_inst) return;
  const Inst in = insts[idx];
  for (int n = threadIdx.x; n <= in.P; n += blockDim.x) {
    const double tau = in.T * (double)n / (double)in.P;
    g[in.state_off + (int64_t)n * in.Nx] = 0.0;
    g[in.state_off + (int64_t)n * in.Nx + in.Nx - 1] = in.Smax - in.K * exp(-in.r * tau);
  }
}

// ---------------------------------------------------------------------------
// Host-side dispatch over the (M, NW) partition classes.
// ---------------------------------------------------------------------------

#define BSP_FOR_EACH_CLASS(X) X(2, 1) X(2, 2) X(2, 4) X(4, 4) X(8, 4) X(16, 4) X(32, 4)

cudaError_t launch_setup(const Inst* d_insts, const int32_t* d_ids, int n, double* pool, double* exptab,
                         cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  setup_kernel<<<dim3(n, 2), 128, 0, s>>>(d_insts, d_ids, pool, exptab);
  return cudaGetLastError();
}

template <typename K>
static cudaError_t set_smem(K kernel, int bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t launch_prop(int M, int NW, bool cn, const PropArgs& a, int n_inst, int maxP, cudaStream_t s) {
  if (n_inst <= 0) return cudaSuccess;
  dim3 grid(maxP, n_inst);
#define X(MM, WW)                                                                \
  if (M == MM && NW == WW) {                                                     \
    const int sz = (int)sizeof(SolverSmem<MM, WW>);                              \
    cudaError_t e;                                                               \
    if (cn) {                                                                    \
      if ((e = set_smem(prop_kernel<MM, WW, true>, sz)) != cudaSuccess) return e;  \
      prop_kernel<MM, WW, true><<<grid, WW * 32, sz, s>>>(a);                    \
    } else {                                                                     \
      if ((e = set_smem(prop_kernel<MM, WW, false>, sz)) != cudaSuccess) return e; \
      prop_kernel<MM, WW, false><<<grid, WW * 32, sz, s>>>(a);                   \
    }                                                                            \
    return cudaGetLastError();                                                   \
  }
  BSP_FOR_EACH_CLASS(X)
#undef X
  return cudaErrorInvalidValue;
}

cudaError_t launch_serial(int M, int NW, const SerialArgs& a, int n_inst, cudaStream_t s) {
  if (n_inst <= 0) return cudaSuccess;
#define X(MM, WW)                                                             \
  if (M == MM && NW == WW) {                                                  \
    const int sz = (int)sizeof(SolverSmem<MM, WW>);                           \
    cudaError_t e = set_smem(serial_fine_kernel<MM, WW>, sz);                 \
    if (e != cudaSuccess) return e;                                           \
    serial_fine_kernel<MM, WW><<<n_inst, WW * 32, sz, s>>>(a);                \
    return cudaGetLastError();                                                \
  }
  BSP_FOR_EACH_CLASS(X)
#undef X
  return cudaErrorInvalidValue;
}

cudaError_t launch_sweep(int M, int NW, const SweepArgs& a, int n_inst, cudaStream_t s) {
  if (n_inst <= 0) return cudaSuccess;
#define X(MM, WW)                                                             \
  if (M == MM && NW == WW) {                                                  \
    const int sz = (int)sizeof(SolverSmem<MM, WW>);                           \
    cudaError_t e = set_smem(sweep_kernel<MM, WW>, sz);                       \
    if (e != cudaSuccess) return e;                                           \
    sweep_kernel<MM, WW><<<n_inst, WW * 32, sz, s>>>(a);                      \
    return cudaGetLastError();                                                \
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
                                     int max_iter, Ctrl* ctrl, double* norms, cudaStream_t s) {
  parareal_finalize_kernel<<<(n_inst + 127) / 128, 128, 0, s>>>(d_insts, n_inst, normbuf, k, tol, max_iter, ctrl,
                                                                norms);
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

cudaError_t launch_table_fix(const Inst* d_insts, int n_inst, double* g, cudaStream_t s) {
  table_fix_kernel<<<n_inst, 64, 0, s>>>(d_insts, n_inst, g);
  return cudaGetLastError();
}

}  // namespace bsp
