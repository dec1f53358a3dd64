// lb_internal.h -- launchers shared between the translation units of the
// library (FP64 parity build, FP32 build, host API).  Not part of the ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace lbk {

template <typename real_t>
struct StepArgs;

// One fused time step fin -> fout.
cudaError_t launch_step(const double *fin, double *fout, const StepArgs<double> &A, cudaStream_t st);
cudaError_t launch_step(const float *fin, float *fout, const StepArgs<float> &A, cudaStream_t st);

// Moments (n, u*) of the stored state; dtype 0 = double, 1 = float outputs.
cudaError_t launch_moments(const double *fin, const StepArgs<double> &A, void *n, void *ux,
                           void *uy, int dtype, cudaStream_t st);
cudaError_t launch_moments(const float *fin, const StepArgs<float> &A, void *n, void *ux,
                           void *uy, int dtype, cudaStream_t st);

// Equilibrium initial state from noise (mode 0) or device fields (mode 1).
cudaError_t launch_init(double *f, int nx, int ny, int mode, uint64_t seed, double rho_mean,
                        double amp, const double *rho0, const double *ux0, const double *uy0,
                        double T, cudaStream_t st);
cudaError_t launch_init(float *f, int nx, int ny, int mode, uint64_t seed, double rho_mean,
                        double amp, const double *rho0, const double *ux0, const double *uy0,
                        double T, cudaStream_t st);

}  // namespace lbk
