// Host-side IMU preintegration for the inertial edges (Eq. 8's r_I; Sec. V-C).
//
// On-manifold preintegration (Forster, Carlone, Dellaert, Scaramuzza, "On-Manifold
// Preintegration for Real-Time Visual-Inertial Odometry", T-RO 2017): between two
// keyframes the gyroscope and accelerometer samples (w_k, a_k), k < n, taken every dt,
// are integrated at fixed bias estimates (bg0, ba0) into relative motion increments
//   dR_{k+1} = dR_k Exp((w_k - bg0) dt)
//   dv_{k+1} = dv_k + dR_k (a_k - ba0) dt
//   dp_{k+1} = dp_k + dv_k dt + dR_k (a_k - ba0) dt^2 / 2,
// together with their first-order Jacobians with respect to the biases (so a later
// bias change is applied without re-integrating) and the covariance of the
// increment errors (dphi, dv, dp), propagated one sample at a time from the discrete
// white-noise covariances sigma_g^2 / dt I and sigma_a^2 / dt I.  This runs once per
// edge when the graph is built; it is not on the per-iteration path.
#include <cmath>
#include <cstring>

#include "gpo.h"

namespace {

using M3 = double[9];

void mat_mul(const double* A, const double* B, double* C, int n, int k, int m) {   // C = A B
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < m; ++j) {
      double s = 0.0;
      for (int t = 0; t < k; ++t) s += A[i * k + t] * B[t * m + j];
      C[i * m + j] = s;
    }
}

void hat(const double* v, double* K) {
  K[0] = 0.0;   K[1] = -v[2]; K[2] = v[1];
  K[3] = v[2];  K[4] = 0.0;   K[5] = -v[0];
  K[6] = -v[1]; K[7] = v[0];  K[8] = 0.0;
}

// Exp(w) = I + a [w]x + b [w]x^2 and Jr(w) = I - b [w]x + c [w]x^2 with a = sin t / t,
// b = (1 - cos t) / t^2, c = (t - sin t) / t^3 (Taylor series below t = 1e-4).
void exp_and_jr(const double* w, double* R, double* Jr) {
  const double t2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  const double t = std::sqrt(t2);
  double a, b, c;
  if (t < 1e-4) {
    a = 1.0 - t2 / 6.0 + t2 * t2 / 120.0;
    b = 0.5 - t2 / 24.0 + t2 * t2 / 720.0;
    c = 1.0 / 6.0 - t2 / 120.0;
  } else {
    a = std::sin(t) / t;
    b = (1.0 - std::cos(t)) / t2;
    c = (t - std::sin(t)) / (t2 * t);
  }
  double K[9], K2[9];
  hat(w, K);
  mat_mul(K, K, K2, 3, 3, 3);
  for (int i = 0; i < 9; ++i) {
    const double I = (i % 4 == 0) ? 1.0 : 0.0;
    R[i] = I + a * K[i] + b * K2[i];
    Jr[i] = I - b * K[i] + c * K2[i];
  }
}

// Inverse of an SPD n x n matrix through its Cholesky factor; false if not SPD.
bool spd_inverse(const double* A, double* Ainv, int n) {
  double L[81] = {}, W[81] = {};
  for (int j = 0; j < n; ++j) {
    double s = A[j * n + j];
    for (int k = 0; k < j; ++k) s -= L[j * n + k] * L[j * n + k];
    if (!(s > 0.0) || !std::isfinite(s)) return false;
    L[j * n + j] = std::sqrt(s);
    for (int i = j + 1; i < n; ++i) {
      double u = A[i * n + j];
      for (int k = 0; k < j; ++k) u -= L[i * n + k] * L[j * n + k];
      L[i * n + j] = u / L[j * n + j];
    }
  }
  for (int i = 0; i < n; ++i) {   // W = L^-1
    W[i * n + i] = 1.0 / L[i * n + i];
    for (int j = 0; j < i; ++j) {
      double u = 0.0;
      for (int k = j; k < i; ++k) u += L[i * n + k] * W[k * n + j];
      W[i * n + j] = -u / L[i * n + i];
    }
  }
  for (int i = 0; i < n; ++i)     // A^-1 = W^T W
    for (int j = 0; j < n; ++j) {
      double u = 0.0;
      for (int k = (i > j ? i : j); k < n; ++k) u += W[k * n + i] * W[k * n + j];
      Ainv[i * n + j] = u;
    }
  return true;
}

}  // namespace

extern "C" gpo_status gpo_imu_preintegrate(const double* gyro, const double* acc, int64_t n, double dt,
                                           const double* bg0, const double* ba0, double sigma_g, double sigma_a,
                                           double* meas_out, double* cov_out, double* info_out) {
  if (!gyro || !acc || !bg0 || !ba0 || !meas_out || n < 1 || !(dt > 0.0) || !(sigma_g > 0.0) || !(sigma_a > 0.0))
    return GPO_ERR_ARG;
  double dR[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, dv[3] = {0, 0, 0}, dp[3] = {0, 0, 0};
  double JRg[9] = {}, Jvg[9] = {}, Jva[9] = {}, Jpg[9] = {}, Jpa[9] = {};
  double cov[81] = {};
  const double qg = sigma_g * sigma_g / dt, qa = sigma_a * sigma_a / dt, dt2 = dt * dt;
  for (int64_t k = 0; k < n; ++k) {
    double w[3], a[3];
    for (int i = 0; i < 3; ++i) {
      w[i] = (gyro[3 * k + i] - bg0[i]) * dt;
      a[i] = acc[3 * k + i] - ba0[i];
    }
    double dRk[9], Jr[9], ah[9], dRah[9];
    exp_and_jr(w, dRk, Jr);
    hat(a, ah);
    mat_mul(dR, ah, dRah, 3, 3, 3);   // dR [a]x
    // error-state transition A (9x9) and noise maps Bg, Ba (9x3)
    double A[81] = {}, Bg[27] = {}, Ba[27] = {};
    for (int i = 0; i < 9; ++i) A[i * 9 + i] = 1.0;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        A[i * 9 + j] = dRk[j * 3 + i];                        // dRk^T
        A[(3 + i) * 9 + j] = -dRah[i * 3 + j] * dt;
        A[(6 + i) * 9 + j] = -0.5 * dRah[i * 3 + j] * dt2;
        Bg[i * 3 + j] = Jr[i * 3 + j] * dt;
        Ba[(3 + i) * 3 + j] = dR[i * 3 + j] * dt;
        Ba[(6 + i) * 3 + j] = 0.5 * dR[i * 3 + j] * dt2;
      }
    for (int i = 0; i < 3; ++i) A[(6 + i) * 9 + 3 + i] = dt;
    // cov <- A cov A^T + qg Bg Bg^T + qa Ba Ba^T
    double T1[81], T2[81];
    mat_mul(A, cov, T1, 9, 9, 9);
    for (int i = 0; i < 9; ++i)
      for (int j = 0; j < 9; ++j) {
        double s = 0.0;
        for (int t = 0; t < 9; ++t) s += T1[i * 9 + t] * A[j * 9 + t];
        double g = 0.0, h = 0.0;
        for (int t = 0; t < 3; ++t) {
          g += Bg[i * 3 + t] * Bg[j * 3 + t];
          h += Ba[i * 3 + t] * Ba[j * 3 + t];
        }
        T2[i * 9 + j] = s + qg * g + qa * h;
      }
    std::memcpy(cov, T2, sizeof(cov));
    // bias Jacobians; the position terms use the previous velocity Jacobians
    double X[9], Y[9];
    mat_mul(dRah, JRg, X, 3, 3, 3);   // dR [a]x JRg
    for (int i = 0; i < 9; ++i) {
      Jpa[i] += Jva[i] * dt - 0.5 * dR[i] * dt2;
      Jpg[i] += Jvg[i] * dt - 0.5 * X[i] * dt2;
      Jva[i] -= dR[i] * dt;
      Jvg[i] -= X[i] * dt;
    }
    // JRg <- dRk^T JRg - Jr dt
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double s = 0.0;
        for (int t = 0; t < 3; ++t) s += dRk[t * 3 + i] * JRg[t * 3 + j];
        Y[i * 3 + j] = s - Jr[i * 3 + j] * dt;
      }
    std::memcpy(JRg, Y, sizeof(JRg));
    // the increments
    double Ra[3];
    for (int i = 0; i < 3; ++i) Ra[i] = dR[3 * i] * a[0] + dR[3 * i + 1] * a[1] + dR[3 * i + 2] * a[2];
    for (int i = 0; i < 3; ++i) {
      dp[i] += dv[i] * dt + 0.5 * Ra[i] * dt2;
      dv[i] += Ra[i] * dt;
    }
    mat_mul(dR, dRk, X, 3, 3, 3);
    std::memcpy(dR, X, sizeof(dR));
  }
  double* m = meas_out;
  std::memcpy(m, dR, 9 * sizeof(double));
  std::memcpy(m + 9, dv, 3 * sizeof(double));
  std::memcpy(m + 12, dp, 3 * sizeof(double));
  std::memcpy(m + 15, JRg, 9 * sizeof(double));
  std::memcpy(m + 24, Jvg, 9 * sizeof(double));
  std::memcpy(m + 33, Jva, 9 * sizeof(double));
  std::memcpy(m + 42, Jpg, 9 * sizeof(double));
  std::memcpy(m + 51, Jpa, 9 * sizeof(double));
  m[60] = dt * (double)n;
  std::memcpy(m + 61, bg0, 3 * sizeof(double));
  std::memcpy(m + 64, ba0, 3 * sizeof(double));
  if (cov_out) std::memcpy(cov_out, cov, sizeof(cov));
  if (info_out && !spd_inverse(cov, info_out, 9)) return GPO_ERR_NUMERIC;
  return GPO_OK;
}
