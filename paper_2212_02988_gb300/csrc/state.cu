// state.cu — single-stream launches of the prediction and of the pose
// matrices; the device bodies are in state_dev.cuh.
#include "state_dev.cuh"

namespace prism {

__global__ void __launch_bounds__(256) k_predict(KParams P, DevState* dev, const double* __restrict__ imu, int n,
                                                 double dt) {
    pdl_enter();
    predict_block(P, dev, imu, n, dt);
}

// The prediction, then (warp 0) the Gauss-Newton start matrices of the new
// prior against the state mean's camera.
__global__ void __launch_bounds__(256) k_predict_prep(KParams P, DevState* dev, const double* __restrict__ imu,
                                                      int n, double dt) {
    pdl_enter();
    predict_block(P, dev, imu, n, dt);
    __syncthreads();
    if (threadIdx.x < 32) {
        PoseArg pa{};
        prep_mats_warp(dev, PREP_REL_NEXT, pa);
    }
}

__global__ void k_prep(DevState* dev, int kind, PoseArg pose) {
    pdl_enter();
    prep_mats_warp(dev, kind, pose);   // one warp
}

cudaError_t launch_prep(DevState* dev, int kind, const PoseArg& pose, cudaStream_t s, bool pdl) {
    if (pdl) return launch_pdl(k_prep, 1, 32, s, dev, kind, pose);
    k_prep<<<1, 32, 0, s>>>(dev, kind, pose);
    return cudaGetLastError();
}

cudaError_t launch_predict(const KParams& P, DevState* dev, const double* imu, int n, double dt, cudaStream_t s,
                           bool pdl) {
    if (pdl) return launch_pdl(k_predict, 1, 256, s, P, dev, imu, n, dt);
    k_predict<<<1, 256, 0, s>>>(P, dev, imu, n, dt);
    return cudaGetLastError();
}

cudaError_t launch_predict_prep(const KParams& P, DevState* dev, const double* imu, int n, double dt,
                                cudaStream_t s) {
    k_predict_prep<<<1, 256, 0, s>>>(P, dev, imu, n, dt);
    return cudaGetLastError();
}

}  // namespace prism
