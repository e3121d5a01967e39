// Superstep kernels instantiated for storage type float2.
#define WSFFT_STORE float2
#define WSFFT_LAUNCH_NAME launch_pass_c32
#include "pass_launch.cuh"
