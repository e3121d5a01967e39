// Ragged-batch kernel instantiated for storage type __half2.
#define WSFFT_STORE __half2
#define WSFFT_RAGGED_NAME launch_ragged_c16f
#include "ragged_launch.cuh"
