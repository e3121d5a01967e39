// Superstep kernels instantiated for storage type __half2.
#define WSFFT_STORE __half2
#define WSFFT_LAUNCH_NAME launch_pass_c16f
#include "pass_launch.cuh"
