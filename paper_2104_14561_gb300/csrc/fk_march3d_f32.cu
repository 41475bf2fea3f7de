// The 3D step of Scheme 1 (kernels in fk_march3d.cuh) in FP32.
#include "fk_march3d.cuh"

template cudaError_t fk_launch_step3d<float>(const Step3D<float>&, cudaStream_t);
template cudaError_t fk_launch_chi3d<float>(const Step3D<float>&, float*, cudaStream_t);
template cudaError_t fk_launch_coef3d<float>(const Step3D<float>&, float*, cudaStream_t);
