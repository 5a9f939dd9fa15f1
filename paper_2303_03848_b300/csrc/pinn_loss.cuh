// pinn_loss.cuh -- per-point pieces of the training loss (Section 3.3,
// Eqs. 11-14) shared by the CUDA-core and tensor-core training kernels.
#pragma once

#include <cmath>

#include "bs_internal.h"

namespace bsp {

// Targets of Eqs. 13-14 and the per-point parameters.
__device__ __forceinline__ void point_setup(const LossArgs& la, int d_in, const double* x, int kind, double& Ki,
                                            double& si, double& ri, double& tgt) {
  Ki = la.K;
  si = la.sigma;
  ri = la.r;
  if (d_in >= 5) {
    si = x[2];
    ri = x[3];
    Ki = x[4];
  }
  const double Sm = (la.smax_over_K > 0.0 && d_in >= 5) ? la.smax_over_K * Ki : la.Smax;
  const double S = x[0], tau = x[1];
  if (kind == 1) tgt = 0.0;
  else if (kind == 2) tgt = Sm - Ki * exp(-ri * tau);
  else if (kind == 3) tgt = S - Ki > 0.0 ? S - Ki : 0.0;
  else tgt = 0.0;
}

// Loss terms and adjoint seeds of one point from its output streams
// (u, u_S, u_SS, u_tau), in FP32 for the tensor-core training path (its outputs
// come from BF16 GEMMs and its seeds are rounded to BF16, so FP32 and the FP32
// exponential carry no error that matters there): kind 0 interior (residual of
// Eq. 1 in tau), 1/2 the S = 0 / S = Smax boundary (Eq. 13), 3 expiry
// (Eq. 14), 4 data point (misfit to its value yv, in term 0; only when the
// call has values, la.y != null).  sq[term] receives the squared error,
// g[4] = dLoss/d(u, u_S, u_SS, u_tau) with each term a mean over its points;
// inv_cnt[term] = 1 / (points of that term).  Any other kind contributes
// nothing (the counting pass records it as an input error).
__device__ __forceinline__ void point_loss_f32(const LossArgs& la, int d_in, const float* x, int kd, float yv,
                                               const float (&out)[4], const float (&inv_cnt)[3], float (&sq)[3],
                                               float (&g)[4]) {
  float Ki = (float)la.K, si = (float)la.sigma, ri = (float)la.r;
  if (d_in >= 5) {
    si = x[2];
    ri = x[3];
    Ki = x[4];
  }
  const float S = x[0];
  g[0] = g[1] = g[2] = g[3] = 0.0f;
  if (kd == 0) {
    const float a = 0.5f * si * si * S * S, b = ri * S;
    const float f = out[3] - a * out[2] - b * out[1] + ri * out[0];
    sq[0] = f * f;
    const float gf = 2.0f * f * inv_cnt[0];
    g[3] = gf;
    g[2] = -a * gf;
    g[1] = -b * gf;
    g[0] = ri * gf;
  } else if (kd == 4 && la.y != nullptr) {
    const float e = out[0] - yv;
    sq[0] = e * e;
    g[0] = 2.0f * e * inv_cnt[0];
  } else if (kd >= 1 && kd <= 3) {
    float tgt = 0.0f;
    if (kd == 2) {
      const float Sm = (la.smax_over_K > 0.0 && d_in >= 5) ? (float)la.smax_over_K * Ki : (float)la.Smax;
      tgt = Sm - Ki * expf(-ri * x[1]);
    } else if (kd == 3) {
      tgt = S - Ki > 0.0f ? S - Ki : 0.0f;
    }
    const float e = out[0] - tgt;
    const int tt = (kd == 3) ? 2 : 1;
    sq[tt] = e * e;
    g[0] = 2.0f * e * inv_cnt[tt];
  }
}

}  // namespace bsp
