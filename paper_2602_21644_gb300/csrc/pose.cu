// FP64 pose step (sm_103a): Adam on the 6-DoF left-perturbation twist of each
// world-to-camera pose, then T <- exp(xi^) T with the closed-form SE(3)
// exponential (Rodrigues' formula and the left Jacobian of SO(3)). FP64
// because the pose's conditioning needs it; one thread per view. The same
// step is fused into the preprocess backward when the tracking loop runs it.
#include "common.cuh"

namespace dags {

namespace {

__global__ void pose_step_kernel(double *__restrict__ poses, const double *__restrict__ grad,
                                 double *__restrict__ state, int views, dags_pose_cfg cfg) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= views) return;
  pose_adam_exp(poses + 12 * v, grad + 6 * v, state + 13 * v, cfg);
}

}  // namespace

cudaError_t launch_pose_step(double *poses, const double *grad, double *state, int views,
                             const dags_pose_cfg &cfg, cudaStream_t s) {
  pose_step_kernel<<<(views + 31) / 32, 32, 0, s>>>(poses, grad, state, views, cfg);
  return cudaGetLastError();
}

}  // namespace dags
