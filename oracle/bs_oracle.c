/*
 * bs_oracle.c -- the ORACLE: plain, serial, FP64 CPU implementation of what the
 * Parareal/PINN hot path computes for the Black-Scholes European call.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant generator with the CUDA library; nothing in the
 * product path may call it.
 *
 * Every routine is written for a reader who checks it against the paper
 * ("Parareal with a physics-informed neural network as coarse propagator",
 * Ibrahim, Goetschel, Ruprecht, arXiv:2303.03848) by eye: no blocking, no
 * fusion, no reordering beyond what the cited passage states.
 *
 * Conventions (readings of the paper where it is silent or ambiguous):
 *  - time-to-maturity tau = T - t, so the terminal condition (Eq. 2) becomes
 *    an initial condition and the solve runs forward in tau (Section 3.2
 *    solves the t-problem backwards from T; this is the same computation);
 *  - grid S_j = j*dS, j = 0..Nx-1, dS = Smax/(Nx-1) (Eq. 9 with N = Nx-1);
 *  - V(tau, 0) = 0 (Eq. 3) and V(tau, Smax) = Smax - K exp(-r tau) (the
 *    far-field reading: the text of Section 3 says the option is worth about
 *    the underlying for large S; Eq. 4 and "V_N = 0" are taken as garbled);
 *  - time slices [tau_n, tau_{n+1}], tau_n = n T / P (Section 3.1).
 *
 * Parity status: every function below is pinned by the CPU test suite
 * (closed-form prices, convergence orders, dense solves, finite
 * differences, hand-computed Adam steps, Parareal invariants).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  double K, sigma, r, T, Smax;
  int32_t Nx, P, fine_steps, coarse_steps;
} orc_params;

/* ------------------------------------------------------------------------ */
/* Problem data: Eq. 2 (payoff), Eq. 3 / far field (Dirichlet values),       */
/* Eq. 10 (semi-discrete operator).                                          */
/* ------------------------------------------------------------------------ */

double orc_dS(const orc_params* p) { return p->Smax / (double)(p->Nx - 1); }

/* Eq. 2 in tau: V(S, tau=0) = max(S - K, 0). */
void orc_payoff(const orc_params* p, double* V) {
  double dS = orc_dS(p);
  for (int j = 0; j < p->Nx; ++j) {
    double S = j * dS;
    V[j] = S - p->K > 0.0 ? S - p->K : 0.0;
  }
}

/* Far-field Dirichlet value at S = Smax (reading of Eq. 4 / Section 3). */
double orc_right_bc(const orc_params* p, double tau) { return p->Smax - p->K * exp(-p->r * tau); }

/*
 * Eq. 10 rewritten in tau (dV/dtau = -dV/dt) with S_j = j dS, so dS cancels:
 *   dV_j/dtau = a_j V_{j-1} + b_j V_j + c_j V_{j+1},
 *   a_j = 1/2 sigma^2 j^2 - 1/2 r j,  b_j = -sigma^2 j^2 - r,  c_j = 1/2 sigma^2 j^2 + 1/2 r j.
 * Arrays have length Nx; entries j = 1..Nx-2 are used.
 */
void orc_coefficients(const orc_params* p, double* a, double* b, double* c) {
  double s2 = p->sigma * p->sigma;
  for (int j = 0; j < p->Nx; ++j) {
    double jj = (double)j;
    a[j] = 0.5 * s2 * jj * jj - 0.5 * p->r * jj;
    b[j] = -s2 * jj * jj - p->r;
    c[j] = 0.5 * s2 * jj * jj + 0.5 * p->r * jj;
  }
}

/*
 * Thomas algorithm (Gaussian elimination without pivoting for a tridiagonal
 * matrix): lo[i] x[i-1] + di[i] x[i] + up[i] x[i+1] = rhs[i], i = 0..n-1.
 * lo[0] and up[n-1] are ignored.  x may alias rhs.  Returns 0, or -1 on a
 * zero pivot or allocation failure.
 */
int orc_thomas(int n, const double* lo, const double* di, const double* up, const double* rhs, double* x) {
  if (n <= 0) return 0;
  double* cp = (double*)malloc(sizeof(double) * (size_t)n);
  double* dp = (double*)malloc(sizeof(double) * (size_t)n);
  if (!cp || !dp) {
    free(cp);
    free(dp);
    return -1;
  }
  double piv = di[0];
  if (piv == 0.0) {
    free(cp);
    free(dp);
    return -1;
  }
  cp[0] = up[0] / piv;
  dp[0] = rhs[0] / piv;
  for (int i = 1; i < n; ++i) {
    piv = di[i] - lo[i] * cp[i - 1];
    if (piv == 0.0) {
      free(cp);
      free(dp);
      return -1;
    }
    cp[i] = up[i] / piv;
    dp[i] = (rhs[i] - lo[i] * dp[i - 1]) / piv;
  }
  x[n - 1] = dp[n - 1];
  for (int i = n - 2; i >= 0; --i) x[i] = dp[i] - cp[i] * x[i + 1];
  free(cp);
  free(dp);
  return 0;
}

/*
 * One Crank-Nicolson step of size dt for the semi-discrete system (Eq. 10),
 * from tau_old = tau_new - dt to tau_new (Section 3.2: CN is the fine method):
 *   (I - dt/2 L) V^{new} = (I + dt/2 L) V^{old} + boundary terms.
 * Interior rows j = 1..Nx-2.  V_0 = 0 at both levels; the old Smax value is
 * taken from V_old[Nx-1], the new one is the Dirichlet value at tau_new.
 */
int orc_cn_step(const orc_params* p, const double* a, const double* b, const double* c, double dt, double tau_new,
                const double* Vold, double* Vnew) {
  int Nx = p->Nx, n = Nx - 2;
  double* lo = (double*)malloc(sizeof(double) * (size_t)n);
  double* di = (double*)malloc(sizeof(double) * (size_t)n);
  double* up = (double*)malloc(sizeof(double) * (size_t)n);
  double* d = (double*)malloc(sizeof(double) * (size_t)n);
  if (!lo || !di || !up || !d) {
    free(lo); free(di); free(up); free(d);
    return -1;
  }
  double Bnew = orc_right_bc(p, tau_new);
  for (int j = 1; j <= Nx - 2; ++j) {
    int i = j - 1;
    /* right-hand side (I + dt/2 L) V^old, including both old boundary values */
    d[i] = 0.5 * dt * a[j] * Vold[j - 1] + (1.0 + 0.5 * dt * b[j]) * Vold[j] + 0.5 * dt * c[j] * Vold[j + 1];
    lo[i] = -0.5 * dt * a[j];
    di[i] = 1.0 - 0.5 * dt * b[j];
    up[i] = -0.5 * dt * c[j];
  }
  /* new-level boundary values move to the right-hand side: V_0^new = 0 adds nothing */
  d[n - 1] += 0.5 * dt * c[Nx - 2] * Bnew;
  int rc = orc_thomas(n, lo, di, up, d, d);
  if (rc == 0) {
    Vnew[0] = 0.0;
    for (int i = 0; i < n; ++i) Vnew[i + 1] = d[i];
    Vnew[Nx - 1] = Bnew;
  }
  free(lo); free(di); free(up); free(d);
  return rc;
}

/*
 * One implicit Euler step of size dt (Section 3.2: IE is the numerical coarse
 * method): (I - dt L) V^{new} = V^{old} + dt c_{Nx-2} V^{new}_{Nx-1} e_last.
 */
int orc_ie_step(const orc_params* p, const double* a, const double* b, const double* c, double dt, double tau_new,
                const double* Vold, double* Vnew) {
  int Nx = p->Nx, n = Nx - 2;
  double* lo = (double*)malloc(sizeof(double) * (size_t)n);
  double* di = (double*)malloc(sizeof(double) * (size_t)n);
  double* up = (double*)malloc(sizeof(double) * (size_t)n);
  double* d = (double*)malloc(sizeof(double) * (size_t)n);
  if (!lo || !di || !up || !d) {
    free(lo); free(di); free(up); free(d);
    return -1;
  }
  double Bnew = orc_right_bc(p, tau_new);
  for (int j = 1; j <= Nx - 2; ++j) {
    int i = j - 1;
    d[i] = Vold[j];
    lo[i] = -dt * a[j];
    di[i] = 1.0 - dt * b[j];
    up[i] = -dt * c[j];
  }
  d[n - 1] += dt * c[Nx - 2] * Bnew;
  int rc = orc_thomas(n, lo, di, up, d, d);
  if (rc == 0) {
    Vnew[0] = 0.0;
    for (int i = 0; i < n; ++i) Vnew[i + 1] = d[i];
    Vnew[Nx - 1] = Bnew;
  }
  free(lo); free(di); free(up); free(d);
  return rc;
}

/* Time of step m (0..M) inside slice n: tau_n + m dtau, written as one product. */
static double slice_time(const orc_params* p, int n, int m, int M) {
  return p->T * (double)((int64_t)n * M + m) / (double)((int64_t)p->P * M);
}

/*
 * The fine propagator F over slice n (Eq. 6): fine_steps CN steps of
 * dtau_f = T / (P * fine_steps) from tau_n to tau_{n+1}.  Vout may alias Vin.
 */
int orc_fine(const orc_params* p, int n, const double* Vin, double* Vout) {
  int Nx = p->Nx, M = p->fine_steps;
  double dt = p->T / ((double)p->P * (double)M);
  double* a = (double*)malloc(sizeof(double) * (size_t)Nx);
  double* b = (double*)malloc(sizeof(double) * (size_t)Nx);
  double* c = (double*)malloc(sizeof(double) * (size_t)Nx);
  double* V = (double*)malloc(sizeof(double) * (size_t)Nx);
  if (!a || !b || !c || !V) {
    free(a); free(b); free(c); free(V);
    return -1;
  }
  orc_coefficients(p, a, b, c);
  memcpy(V, Vin, sizeof(double) * (size_t)Nx);
  int rc = 0;
  for (int m = 0; m < M && rc == 0; ++m) rc = orc_cn_step(p, a, b, c, dt, slice_time(p, n, m + 1, M), V, V);
  memcpy(Vout, V, sizeof(double) * (size_t)Nx);
  free(a); free(b); free(c); free(V);
  return rc;
}

/* The numerical coarse propagator G over slice n: coarse_steps IE steps. */
int orc_coarse_ie(const orc_params* p, int n, const double* Vin, double* Vout) {
  int Nx = p->Nx, M = p->coarse_steps;
  double dt = p->T / ((double)p->P * (double)M);
  double* a = (double*)malloc(sizeof(double) * (size_t)Nx);
  double* b = (double*)malloc(sizeof(double) * (size_t)Nx);
  double* c = (double*)malloc(sizeof(double) * (size_t)Nx);
  double* V = (double*)malloc(sizeof(double) * (size_t)Nx);
  if (!a || !b || !c || !V) {
    free(a); free(b); free(c); free(V);
    return -1;
  }
  orc_coefficients(p, a, b, c);
  memcpy(V, Vin, sizeof(double) * (size_t)Nx);
  int rc = 0;
  for (int m = 0; m < M && rc == 0; ++m) rc = orc_ie_step(p, a, b, c, dt, slice_time(p, n, m + 1, M), V, V);
  memcpy(Vout, V, sizeof(double) * (size_t)Nx);
  free(a); free(b); free(c); free(V);
  return rc;
}

/* Classical serial time stepping, Eq. 6 for n = 0..P-1: U[0] = payoff, U[n+1] = F(U[n]). */
int orc_serial_fine(const orc_params* p, double* U) {
  int Nx = p->Nx;
  orc_payoff(p, U);
  for (int n = 0; n < p->P; ++n) {
    int rc = orc_fine(p, n, U + (size_t)n * Nx, U + (size_t)(n + 1) * Nx);
    if (rc) return rc;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Parareal, Eq. 7 (Section 3.1).                                            */
/* ------------------------------------------------------------------------ */

enum { ORC_COARSE_IE = 0, ORC_COARSE_PINN = 1, ORC_COARSE_PINN_INCR = 2, ORC_COARSE_PINN_IE = 3 };

/*
 * The coarse propagator G over slice n applied to V.
 *   IE:        coarse_steps implicit Euler steps (Section 3.2).
 *   PINN:      the network's prediction at tau_{n+1} on the grid, g[n+1]
 *              (Section 3.3 trains V~(t, S) only, so G does not depend on V).
 *   PINN_INCR: V + g[n+1] - g[n] (a state-dependent use of the same network).
 *   PINN_IE:   the network's prediction at tau_{n+1} plus the implicit Euler
 *              response to the deviation of V from the network's value at
 *              tau_n (Section 3.3 / Fig. 2: the network is given V at
 *              t_start).  IE is affine, IE(V) = A^{-1}(V + boundary terms),
 *              so g[n+1] + A^{-1}(V - g[n]) is written as
 *                 IE(V) + (g[n+1] - IE(g[n]))
 *              at the interior nodes; the Dirichlet nodes are IE's exact values.
 *              When V = g[n] it returns g[n+1]: the network's own solution is a
 *              trajectory of this G.
 * g holds (P+1) x Nx network values whose Dirichlet nodes already carry the
 * exact boundary values.
 */
static int coarse_apply(const orc_params* p, int kind, const double* g, int n, const double* V, double* out) {
  int Nx = p->Nx;
  if (kind == ORC_COARSE_IE) return orc_coarse_ie(p, n, V, out);
  if (kind == ORC_COARSE_PINN) {
    memcpy(out, g + (size_t)(n + 1) * Nx, sizeof(double) * (size_t)Nx);
    return 0;
  }
  if (kind == ORC_COARSE_PINN_INCR) {
    for (int j = 0; j < Nx; ++j) out[j] = V[j] + (g[(size_t)(n + 1) * Nx + j] - g[(size_t)n * Nx + j]);
    return 0;
  }
  if (kind == ORC_COARSE_PINN_IE) {
    double* gie = (double*)malloc(sizeof(double) * (size_t)Nx);
    if (!gie) return -1;
    int rc = orc_coarse_ie(p, n, V, out);
    if (rc == 0) rc = orc_coarse_ie(p, n, g + (size_t)n * Nx, gie);
    if (rc == 0)
      for (int j = 1; j <= Nx - 2; ++j) out[j] = out[j] + (g[(size_t)(n + 1) * Nx + j] - gie[j]);
    free(gie);
    return rc;
  }
  return -1;
}

static double l2(const double* x, int n) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += x[i] * x[i];
  return sqrt(s);
}

/*
 * Parareal (Eq. 7): U^{k+1}_{n+1} = G(U^{k+1}_n) + F(U^k_n) - G(U^k_n),
 * evaluated as F + (G_new - G_old) so that a slice whose start value no longer
 * changes reproduces the serial fine value exactly.
 *
 * Iteration k (0-based) runs F on slices n >= k only: slices n < k start from
 * values that equal the serial fine ones (Section 3.1: after k iterations the
 * first k slices are exact), so their F would reproduce U^k_{n+1}.
 * Stop rule: increment norm e_k = max_n ||U^{k+1}_n - U^k_n||_2 / ||U^{k+1}_n||_2 <= tol,
 * or k + 1 == P (Parareal then equals serial fine), or k + 1 == max_iter.
 *
 * U: (P+1) x Nx output.  norms: max_iter increment norms.  *iters: iterations
 * done.  Returns 0 converged (or exact at k = P), 1 max_iter reached, 2 a
 * non-finite norm, <0 error.
 */
int orc_parareal(const orc_params* p, int kind, const double* g, double tol, int max_iter, double* U, double* norms,
                 int* iters) {
  int Nx = p->Nx, P = p->P;
  size_t sz = (size_t)(P + 1) * Nx;
  double* Unew = (double*)malloc(sizeof(double) * sz);
  double* Fv = (double*)malloc(sizeof(double) * (size_t)P * Nx);
  double* Gold = (double*)malloc(sizeof(double) * (size_t)P * Nx);
  double* Gnew = (double*)malloc(sizeof(double) * (size_t)Nx);
  double* diff = (double*)malloc(sizeof(double) * (size_t)Nx);
  int status = -1, rc = 0;
  *iters = 0;
  if (!Unew || !Fv || !Gold || !Gnew || !diff) goto done;
  /* initial coarse sweep: U^0_0 = payoff, U^0_{n+1} = G(U^0_n) */
  orc_payoff(p, U);
  for (int n = 0; n < P; ++n) {
    rc = coarse_apply(p, kind, g, n, U + (size_t)n * Nx, Gold + (size_t)n * Nx);
    if (rc) goto done;
    memcpy(U + (size_t)(n + 1) * Nx, Gold + (size_t)n * Nx, sizeof(double) * (size_t)Nx);
  }
  status = 1;
  for (int k = 0; k < max_iter; ++k) {
    /* fine propagation, parallel across slices in the paper */
    for (int n = k; n < P; ++n) {
      rc = orc_fine(p, n, U + (size_t)n * Nx, Fv + (size_t)n * Nx);
      if (rc) { status = -1; goto done; }
    }
    /* serial coarse sweep with correction */
    memcpy(Unew, U, sizeof(double) * (size_t)(k + 1) * Nx);
    for (int n = k; n < P; ++n) {
      rc = coarse_apply(p, kind, g, n, Unew + (size_t)n * Nx, Gnew);
      if (rc) { status = -1; goto done; }
      for (int j = 0; j < Nx; ++j) {
        Unew[(size_t)(n + 1) * Nx + j] = Fv[(size_t)n * Nx + j] + (Gnew[j] - Gold[(size_t)n * Nx + j]);
        Gold[(size_t)n * Nx + j] = Gnew[j];
      }
    }
    /* increment norm */
    double e = 0.0;
    int bad = 0;
    for (int n = 1; n <= P; ++n) {
      for (int j = 0; j < Nx; ++j) diff[j] = Unew[(size_t)n * Nx + j] - U[(size_t)n * Nx + j];
      double num = l2(diff, Nx), den = l2(Unew + (size_t)n * Nx, Nx);
      double q = den > 0.0 ? num / den : num;
      if (!(q == q) || isinf(q)) bad = 1;
      if (q > e) e = q;
    }
    memcpy(U, Unew, sizeof(double) * sz);
    norms[k] = bad ? NAN : e;
    *iters = k + 1;
    if (bad) { status = 2; break; }
    if (e <= tol || k + 1 >= P) { status = 0; break; }
  }
done:
  free(Unew); free(Fv); free(Gold); free(Gnew); free(diff);
  return status;
}

/* Normalized l2 error of U against a reference, max over slices 1..P (Fig. 3 measure). */
double orc_rel_error(const orc_params* p, const double* U, const double* Uref) {
  int Nx = p->Nx;
  double e = 0.0;
  for (int n = 1; n <= p->P; ++n) {
    double num = 0.0, den = 0.0;
    for (int j = 0; j < Nx; ++j) {
      double d = U[(size_t)n * Nx + j] - Uref[(size_t)n * Nx + j];
      num += d * d;
      den += Uref[(size_t)n * Nx + j] * Uref[(size_t)n * Nx + j];
    }
    double q = den > 0.0 ? sqrt(num / den) : sqrt(num);
    if (q > e) e = q;
  }
  return e;
}

/* Speedup bound, Eq. 8. */
double orc_speedup_bound(int P, int K, double cc_over_cf) {
  return 1.0 / ((1.0 + (double)K / P) * cc_over_cf + (double)K / P);
}

/* Closed-form price of a European call (Section 3 cites its existence):
 * V = S N(d1) - K e^{-r tau} N(d2), N(x) = erfc(-x/sqrt 2)/2. */
double orc_bs_call(double S, double K, double r, double sigma, double tau) {
  if (tau <= 0.0) return S - K > 0.0 ? S - K : 0.0;
  if (S <= 0.0) return 0.0;
  double sq = sigma * sqrt(tau);
  double d1 = (log(S / K) + (r + 0.5 * sigma * sigma) * tau) / sq;
  double d2 = d1 - sq;
  return S * 0.5 * erfc(-d1 / sqrt(2.0)) - K * exp(-r * tau) * 0.5 * erfc(-d2 / sqrt(2.0));
}

/* ------------------------------------------------------------------------ */
/* PINN (Section 3.3): fully connected tanh network in (S, tau).             */
/* ------------------------------------------------------------------------ */
/*
 * Model definition (both sides follow this written contract, no shared code):
 *   widths[0..n_lin]: widths[0] = d_in (2: (S, tau); 5: (S, tau, sigma, r, K)),
 *   widths[n_lin] = 1.  Linear layer l (1..n_lin) maps widths[l-1] -> widths[l];
 *   params hold, per layer, W_l row-major [w_out][w_in] then b_l [w_out].
 *   Input map x^_i = 2 (x_i - lo_i) / (hi_i - lo_i) - 1.
 *   Hidden layers h_l = tanh(W_l h_{l-1} + b_l); the output layer is linear.
 * Derivatives u_S, u_SS, u_tau (Section 3.3 takes them by automatic
 * differentiation): forward-mode chain rule through each layer,
 *   z' = W h',  h' = (1 - h^2) z',  h'' = (1 - h^2) z'' - 2 h (1 - h^2) (z')^2.
 */

static int64_t n_params_of(int n_lin, const int32_t* w) {
  int64_t s = 0;
  for (int l = 1; l <= n_lin; ++l) s += (int64_t)w[l] * w[l - 1] + w[l];
  return s;
}

int64_t orc_mlp_n_params(int n_lin, const int32_t* widths) { return n_params_of(n_lin, widths); }

static int max_width(int n_lin, const int32_t* w) {
  int m = 0;
  for (int l = 0; l <= n_lin; ++l)
    if (w[l] > m) m = w[l];
  return m;
}

/*
 * Forward pass for one point with the derivative streams (S = input 0,
 * tau = input 1).  Stores, if acts != NULL, per hidden layer l the values
 * needed by the adjoint: t = tanh(z), z_S, z_SS, z_tau (each widths[l]).
 * out[0..3] = u, u_S, u_SS, u_tau.
 */
static void mlp_point(int n_lin, const int32_t* w, const double* prm, const double* lo, const double* hi,
                      const double* x, double* out, double* h, double* hS, double* hSS, double* hT, double* z,
                      double* zS, double* zSS, double* zT, double* acts) {
  int d_in = w[0];
  for (int i = 0; i < d_in; ++i) {
    double sc = 2.0 / (hi[i] - lo[i]);
    h[i] = sc * (x[i] - lo[i]) - 1.0;
    hS[i] = (i == 0) ? sc : 0.0;
    hSS[i] = 0.0;
    hT[i] = (i == 1) ? sc : 0.0;
  }
  const double* P = prm;
  size_t aoff = 0;
  for (int l = 1; l <= n_lin; ++l) {
    int wi = w[l - 1], wo = w[l];
    const double* W = P;
    const double* b = P + (size_t)wo * wi;
    for (int o = 0; o < wo; ++o) {
      double s = b[o], sS = 0.0, sSS = 0.0, sT = 0.0;
      for (int i = 0; i < wi; ++i) {
        double wv = W[(size_t)o * wi + i];
        s += wv * h[i];
        sS += wv * hS[i];
        sSS += wv * hSS[i];
        sT += wv * hT[i];
      }
      z[o] = s;
      zS[o] = sS;
      zSS[o] = sSS;
      zT[o] = sT;
    }
    if (l < n_lin) {
      for (int o = 0; o < wo; ++o) {
        double t = tanh(z[o]);
        double d1 = 1.0 - t * t;
        h[o] = t;
        hS[o] = d1 * zS[o];
        hSS[o] = d1 * zSS[o] - 2.0 * t * d1 * zS[o] * zS[o];
        hT[o] = d1 * zT[o];
        if (acts) {
          acts[aoff + o] = t;
          acts[aoff + wo + o] = zS[o];
          acts[aoff + 2 * (size_t)wo + o] = zSS[o];
          acts[aoff + 3 * (size_t)wo + o] = zT[o];
        }
      }
      aoff += 4 * (size_t)wo;
    } else {
      out[0] = z[0];
      out[1] = zS[0];
      out[2] = zSS[0];
      out[3] = zT[0];
    }
    P += (size_t)wo * wi + wo;
  }
}

/* Evaluate the network at N points X[N][d_in]: u[N] and, if derivs != NULL, derivs[N][3] = (u_S, u_SS, u_tau). */
int orc_mlp_eval(int n_lin, const int32_t* widths, const double* params, const double* lo, const double* hi,
                 const double* X, int64_t N, double* u, double* derivs) {
  int mw = max_width(n_lin, widths);
  double* buf = (double*)malloc(sizeof(double) * 8 * (size_t)mw);
  if (!buf) return -1;
  double out[4];
  for (int64_t k = 0; k < N; ++k) {
    mlp_point(n_lin, widths, params, lo, hi, X + k * widths[0], out, buf, buf + mw, buf + 2 * mw, buf + 3 * mw,
              buf + 4 * mw, buf + 5 * mw, buf + 6 * mw, buf + 7 * mw, NULL);
    u[k] = out[0];
    if (derivs) {
      derivs[3 * k + 0] = out[1];
      derivs[3 * k + 1] = out[2];
      derivs[3 * k + 2] = out[3];
    }
  }
  free(buf);
  return 0;
}

/*
 * The coarse-propagator table of the state-independent network coarse
 * propagator: g[n][j] = u_theta(S_j, tau_n) for n = 0..P, j = 0..Nx-1, with the
 * Dirichlet nodes replaced by the exact values (Eq. 3 and the far-field
 * value).  A 5-input network receives (S, tau, sigma, r, K).
 */
int orc_pinn_table(const orc_params* p, int n_lin, const int32_t* widths, const double* params, const double* lo,
                   const double* hi, double* g) {
  int Nx = p->Nx, d_in = widths[0];
  double dS = orc_dS(p);
  double x[8];
  for (int n = 0; n <= p->P; ++n) {
    double tau = p->T * (double)n / (double)p->P;
    for (int j = 0; j < Nx; ++j) {
      x[0] = j * dS;
      x[1] = tau;
      if (d_in >= 5) {
        x[2] = p->sigma;
        x[3] = p->r;
        x[4] = p->K;
      }
      if (orc_mlp_eval(n_lin, widths, params, lo, hi, x, 1, g + (size_t)n * Nx + j, NULL)) return -1;
    }
    g[(size_t)n * Nx] = 0.0;
    g[(size_t)n * Nx + Nx - 1] = orc_right_bc(p, tau);
  }
  return 0;
}

/*
 * Collocation kinds: 0 interior (residual, Eq. 12), 1 boundary S = 0 and
 * 2 boundary S = Smax (Eq. 13, both in one mean), 3 expiry tau = 0 (Eq. 14),
 * 4 data point: squared misfit (u - y)^2 to a given value y, in the mean of
 * term 0 (Section 4 trains a network on fine-propagator output alone, without
 * the PDE terms, for comparison with the PINN).  Any other kind, or a data
 * point when no values y are given, is an input error (return -2).
 * Residual in tau: f = u_tau - 1/2 sigma^2 S^2 u_SS - r S u_S + r u (Eq. 1 with
 * dV/dt = -dV/dtau, sign flipped; |f|^2 is unchanged).  The sigma, r, K used in
 * the residual and targets are the ones given here (a parametric network also
 * receives them as inputs 2..4, taken from X).
 */
static void point_targets(int kind, const double* x, int d_in, double K, double sigma, double r, double Smax,
                          double* Kp, double* sp, double* rp, double* target) {
  double Ki = K, si = sigma, ri = r;
  if (d_in >= 5) {
    si = x[2];
    ri = x[3];
    Ki = x[4];
  }
  *Kp = Ki;
  *sp = si;
  *rp = ri;
  double S = x[0], tau = x[1];
  if (kind == 1) *target = 0.0;
  else if (kind == 2) *target = Smax - Ki * exp(-ri * tau);
  else if (kind == 3) *target = S - Ki > 0.0 ? S - Ki : 0.0;
  else *target = 0.0;
}

/*
 * Total loss, Eq. 11 = MSE_f (Eq. 12) + MSE_exp (Eq. 14) + MSE_b (Eq. 13),
 * each the mean over its own points.  terms[0..2] = MSE_f, MSE_b, MSE_exp.
 * If grad != NULL, also the gradient of the total with respect to params,
 * by reverse-mode differentiation of mlp_point (written out by hand).
 * For a parametric net the Smax of the S = Smax points is K-relative:
 * Smax_i = smax_over_K * K_i when smax_over_K > 0, else Smax.
 */
int orc_pinn_loss_grad_y(int n_lin, const int32_t* w, const double* params, const double* lo, const double* hi,
                         const double* X, const int8_t* kind, const double* y, int64_t N, double K, double sigma,
                         double r, double Smax, double smax_over_K, double* terms, double* grad) {
  int d_in = w[0];
  int mw = max_width(n_lin, w);
  int64_t np_ = n_params_of(n_lin, w);
  size_t act_sz = 0;
  for (int l = 1; l < n_lin; ++l) act_sz += 4 * (size_t)w[l];
  double* buf = (double*)malloc(sizeof(double) * 8 * (size_t)mw);
  double* acts = (double*)malloc(sizeof(double) * (act_sz + 1));
  double* adj = (double*)malloc(sizeof(double) * 8 * (size_t)mw);
  double* x0 = (double*)malloc(sizeof(double) * 4 * (size_t)d_in);
  if (!buf || !acts || !adj || !x0 || n_lin > 63) {
    free(buf); free(acts); free(adj); free(x0);
    return -1;
  }
  int64_t poff[64];
  {
    int64_t o = 0;
    for (int l = 1; l <= n_lin; ++l) {
      poff[l] = o;
      o += (int64_t)w[l] * w[l - 1] + w[l];
    }
  }
  int64_t cnt[3] = {0, 0, 0};
  for (int64_t k = 0; k < N; ++k) {
    if (kind[k] == 0 || (kind[k] == 4 && y)) cnt[0]++;
    else if (kind[k] == 1 || kind[k] == 2) cnt[1]++;
    else if (kind[k] == 3) cnt[2]++;
    else {  /* a kind outside 0..3, or a data point without its value */
      free(buf); free(acts); free(adj); free(x0);
      return -2;
    }
  }
  double sums[3] = {0.0, 0.0, 0.0};
  if (grad) memset(grad, 0, sizeof(double) * (size_t)np_);
  double out[4];
  for (int64_t k = 0; k < N; ++k) {
    const double* x = X + k * d_in;
    double Ki, si, ri, tgt;
    double Sm = (smax_over_K > 0.0 && d_in >= 5) ? smax_over_K * x[4] : Smax;
    point_targets(kind[k], x, d_in, K, sigma, r, Sm, &Ki, &si, &ri, &tgt);
    mlp_point(n_lin, w, params, lo, hi, x, out, buf, buf + mw, buf + 2 * mw, buf + 3 * mw, buf + 4 * mw,
              buf + 5 * mw, buf + 6 * mw, buf + 7 * mw, acts);
    double S = x[0];
    /* seeds: dLoss/d(u, u_S, u_SS, u_tau) for this point */
    double gu = 0.0, gS = 0.0, gSS = 0.0, gT = 0.0;
    if (kind[k] == 0) {
      double f = out[3] - 0.5 * si * si * S * S * out[2] - ri * S * out[1] + ri * out[0];
      sums[0] += f * f;
      double gf = 2.0 * f / (double)cnt[0];
      gT = gf;
      gSS = -0.5 * si * si * S * S * gf;
      gS = -ri * S * gf;
      gu = ri * gf;
    } else if (kind[k] == 4) {
      double e = out[0] - y[k];
      sums[0] += e * e;
      gu = 2.0 * e / (double)cnt[0];
    } else {
      double e = out[0] - tgt;
      int t = (kind[k] == 3) ? 2 : 1;
      sums[t] += e * e;
      gu = 2.0 * e / (double)cnt[t];
    }
    if (!grad) continue;
    /* reverse sweep; adjoints of the current layer's input streams and of z */
    double* ah = adj;
    double* ahS = adj + mw;
    double* ahSS = adj + 2 * mw;
    double* ahT = adj + 3 * mw;
    double* az = adj + 4 * mw;
    double* azS = adj + 5 * mw;
    double* azSS = adj + 6 * mw;
    double* azT = adj + 7 * mw;
    /* output layer: its z is the output, so dz = seeds */
    az[0] = gu;
    azS[0] = gS;
    azSS[0] = gSS;
    azT[0] = gT;
    size_t aoff_end = act_sz;
    for (int l = n_lin; l >= 1; --l) {
      int wi = w[l - 1], wo = w[l];
      const double* W = params + poff[l];
      double* gW = grad + poff[l];
      double* gb = gW + (size_t)wo * wi;
      /* input streams of layer l: h_{l-1} (rebuilt from stored t, z'), or the input map for l = 1 */
      const double *hin, *hSin, *hSSin, *hTin;
      if (l > 1) {
        size_t a0 = aoff_end - 4 * (size_t)wi;
        const double* t = acts + a0;
        const double* zs = acts + a0 + wi;
        const double* zss = acts + a0 + 2 * (size_t)wi;
        const double* zt = acts + a0 + 3 * (size_t)wi;
        for (int i = 0; i < wi; ++i) {
          double d1 = 1.0 - t[i] * t[i];
          buf[i] = t[i];
          buf[mw + i] = d1 * zs[i];
          buf[2 * mw + i] = d1 * zss[i] - 2.0 * t[i] * d1 * zs[i] * zs[i];
          buf[3 * mw + i] = d1 * zt[i];
        }
        hin = buf;
        hSin = buf + mw;
        hSSin = buf + 2 * mw;
        hTin = buf + 3 * mw;
      } else {
        for (int i = 0; i < d_in; ++i) {
          double sc = 2.0 / (hi[i] - lo[i]);
          x0[i] = sc * (x[i] - lo[i]) - 1.0;
          x0[d_in + i] = (i == 0) ? sc : 0.0;
          x0[2 * d_in + i] = 0.0;
          x0[3 * d_in + i] = (i == 1) ? sc : 0.0;
        }
        hin = x0;
        hSin = x0 + d_in;
        hSSin = x0 + 2 * d_in;
        hTin = x0 + 3 * d_in;
      }
      /* parameter gradients: z = W h + b, z_S = W h_S, z_SS = W h_SS, z_tau = W h_tau */
      for (int o = 0; o < wo; ++o) {
        gb[o] += az[o];
        for (int i = 0; i < wi; ++i)
          gW[(size_t)o * wi + i] += az[o] * hin[i] + azS[o] * hSin[i] + azSS[o] * hSSin[i] + azT[o] * hTin[i];
      }
      if (l == 1) break;
      /* adjoints of the input streams: W^T dz */
      for (int i = 0; i < wi; ++i) {
        double s = 0.0, sS = 0.0, sSS = 0.0, sT = 0.0;
        for (int o = 0; o < wo; ++o) {
          double wv = W[(size_t)o * wi + i];
          s += wv * az[o];
          sS += wv * azS[o];
          sSS += wv * azSS[o];
          sT += wv * azT[o];
        }
        ah[i] = s;
        ahS[i] = sS;
        ahSS[i] = sSS;
        ahT[i] = sT;
      }
      /* back through the tanh of layer l-1:
       *   h = t, h_S = t' z_S, h_SS = t' z_SS + t'' z_S^2, h_tau = t' z_tau,
       *   t' = 1 - t^2, t'' = -2 t t'. */
      size_t a0 = aoff_end - 4 * (size_t)wi;
      const double* t = acts + a0;
      const double* zs = acts + a0 + wi;
      const double* zss = acts + a0 + 2 * (size_t)wi;
      const double* zt = acts + a0 + 3 * (size_t)wi;
      for (int i = 0; i < wi; ++i) {
        double tv = t[i], d1 = 1.0 - tv * tv, d2 = -2.0 * tv * d1;
        double bar_d1 = ahS[i] * zs[i] + ahSS[i] * zss[i] + ahT[i] * zt[i];
        double bar_d2 = ahSS[i] * zs[i] * zs[i];
        double bar_t = ah[i];
        bar_t += -2.0 * d1 * bar_d2;  /* d2 = -2 t d1 */
        bar_d1 += -2.0 * tv * bar_d2;
        bar_t += -2.0 * tv * bar_d1;  /* d1 = 1 - t^2 */
        az[i] = d1 * bar_t;           /* t = tanh(z) */
        azS[i] = ahS[i] * d1 + 2.0 * ahSS[i] * d2 * zs[i];
        azSS[i] = ahSS[i] * d1;
        azT[i] = ahT[i] * d1;
      }
      aoff_end = a0;
    }
  }
  terms[0] = cnt[0] ? sums[0] / (double)cnt[0] : 0.0;
  terms[1] = cnt[1] ? sums[1] / (double)cnt[1] : 0.0;
  terms[2] = cnt[2] ? sums[2] / (double)cnt[2] : 0.0;
  free(buf); free(acts); free(adj); free(x0);
  return 0;
}

/* The PINN loss alone (no data points). */
int orc_pinn_loss_grad(int n_lin, const int32_t* w, const double* params, const double* lo, const double* hi,
                       const double* X, const int8_t* kind, int64_t N, double K, double sigma, double r, double Smax,
                       double smax_over_K, double* terms, double* grad) {
  return orc_pinn_loss_grad_y(n_lin, w, params, lo, hi, X, kind, NULL, N, K, sigma, r, Smax, smax_over_K, terms,
                              grad);
}

/*
 * One Adam step (Section 3.3 trains with Adam; Kingma & Ba's update):
 *   m = b1 m + (1-b1) g,  v = b2 v + (1-b2) g^2,
 *   theta -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps),  t = step (1-based).
 */
void orc_adam(int64_t n, double* theta, double* m, double* v, const double* g, int t, double lr, double b1, double b2,
              double eps) {
  double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
  for (int64_t i = 0; i < n; ++i) {
    m[i] = b1 * m[i] + (1.0 - b1) * g[i];
    v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
    double mh = m[i] / c1, vh = v[i] / c2;
    theta[i] -= lr * mh / (sqrt(vh) + eps);
  }
}
