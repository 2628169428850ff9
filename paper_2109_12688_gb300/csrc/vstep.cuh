// Closed-form v-step of the ADMM iteration (Eq. 5 line 1, Eq. 6), shared by
// the pass kernels.
#pragma once
#include "fft_device.cuh"

namespace nadmm {

// s = 2 (Eq. 6 middle, Sherman-Morrison): v = u - rho(u) J / (theta + |J|^2)
// s = 1 (Eq. 6 top):  z = theta rho(u) / (|J|^2 + eps),
//                     v = u - z / max(|z|, 1) * J / theta
// with rho(u) = J . u + c.
NADMM_HD void v_step(int data_term, float theta, float eps, const float (&J)[3], float c,
                     const float (&u)[3], float (&v)[3]) {
  float rho = J[0] * u[0] + J[1] * u[1] + J[2] * u[2] + c;
  float jj = J[0] * J[0] + J[1] * J[1] + J[2] * J[2];
  float f;
  if (data_term == 2) {
    f = rho / (theta + jj);
  } else {
    float z = theta * rho / (jj + eps);
    float t = z / fmaxf(fabsf(z), 1.0f);
    f = t / theta;
  }
  v[0] = u[0] - f * J[0];
  v[1] = u[1] - f * J[1];
  v[2] = u[2] - f * J[2];
}

}  // namespace nadmm
