// FP64 pose step (sm_103a): Adam on the 6-DoF left-perturbation twist of each
// world-to-camera pose, then T <- exp(xi^) T with the closed-form SE(3)
// exponential (Rodrigues' formula and the left Jacobian of SO(3); series
// forms below |phi| = 1e-4). FP64 because the pose's conditioning needs it;
// one thread per view, negligible time.
#include "common.cuh"

namespace dags {

namespace {

__global__ void pose_step_kernel(double *__restrict__ poses, const double *__restrict__ grad,
                                 double *__restrict__ state, int views, dags_pose_cfg cfg) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= views) return;
  double *st = state + 13 * v;
  const double k = st[12] + 1.0;
  const double bc1 = 1.0 - pow(cfg.beta1, k), bc2 = 1.0 - pow(cfg.beta2, k);
  double xi[6];
  for (int c = 0; c < 6; ++c) {
    const double g = grad[6 * v + c];
    const double m = cfg.beta1 * st[c] + (1.0 - cfg.beta1) * g;
    const double s2 = cfg.beta2 * st[6 + c] + (1.0 - cfg.beta2) * g * g;
    st[c] = m;
    st[6 + c] = s2;
    xi[c] = -cfg.lr[c] * (m / bc1) / (sqrt(s2 / bc2) + cfg.eps);
  }
  st[12] = k;
  const double px = xi[3], py = xi[4], pz = xi[5];
  const double th2 = px * px + py * py + pz * pz;
  double a, b, c;
  if (th2 < 1e-8) {
    a = 1.0 - th2 / 6.0;
    b = 0.5 - th2 / 24.0;
    c = 1.0 / 6.0 - th2 / 120.0;
  } else {
    const double th = sqrt(th2);
    a = sin(th) / th;
    b = (1.0 - cos(th)) / th2;
    c = (th - sin(th)) / (th2 * th);
  }
  // hat(phi) and its square
  const double Kh[9] = {0.0, -pz, py, pz, 0.0, -px, -py, px, 0.0};
  double K2[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      K2[3 * i + j] = Kh[3 * i] * Kh[j] + Kh[3 * i + 1] * Kh[3 + j] + Kh[3 * i + 2] * Kh[6 + j];
  double Re[9], V[9];
  for (int e = 0; e < 9; ++e) {
    const double I = (e % 4 == 0) ? 1.0 : 0.0;
    Re[e] = I + a * Kh[e] + b * K2[e];
    V[e] = I + b * Kh[e] + c * K2[e];
  }
  double te[3];
  for (int i = 0; i < 3; ++i) te[i] = V[3 * i] * xi[0] + V[3 * i + 1] * xi[1] + V[3 * i + 2] * xi[2];
  double *T = poses + 12 * v;
  double out[12];
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j)
      out[4 * i + j] = Re[3 * i] * T[j] + Re[3 * i + 1] * T[4 + j] + Re[3 * i + 2] * T[8 + j];
    out[4 * i + 3] = Re[3 * i] * T[3] + Re[3 * i + 1] * T[7] + Re[3 * i + 2] * T[11] + te[i];
  }
  for (int e = 0; e < 12; ++e) T[e] = out[e];
}

}  // namespace

cudaError_t launch_pose_step(double *poses, const double *grad, double *state, int views,
                             const dags_pose_cfg &cfg, cudaStream_t s) {
  pose_step_kernel<<<(views + 31) / 32, 32, 0, s>>>(poses, grad, state, views, cfg);
  return cudaGetLastError();
}

}  // namespace dags
