// Ragged-batch kernel instantiated for storage type __nv_bfloat162.
#define WSFFT_STORE __nv_bfloat162
#define WSFFT_RAGGED_NAME launch_ragged_c16bf
#include "ragged_launch.cuh"
