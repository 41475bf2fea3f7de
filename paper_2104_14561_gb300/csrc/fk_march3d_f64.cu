// The 3D step of Scheme 1 (kernels in fk_march3d.cuh) in FP64.
#include "fk_march3d.cuh"

template cudaError_t fk_launch_step3d<double>(const Step3D<double>&, cudaStream_t);
template cudaError_t fk_launch_chi3d<double>(const Step3D<double>&, double*, cudaStream_t);
template cudaError_t fk_launch_coef3d<double>(const Step3D<double>&, double*, cudaStream_t);
