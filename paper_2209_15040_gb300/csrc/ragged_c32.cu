// Ragged-batch kernel instantiated for storage type float2.
#define WSFFT_STORE float2
#define WSFFT_RAGGED_NAME launch_ragged_c32
#include "ragged_launch.cuh"
