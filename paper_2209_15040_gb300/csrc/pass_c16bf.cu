// Superstep kernels instantiated for storage type __nv_bfloat162.
#define WSFFT_STORE __nv_bfloat162
#define WSFFT_LAUNCH_NAME launch_pass_c16bf
#include "pass_launch.cuh"
