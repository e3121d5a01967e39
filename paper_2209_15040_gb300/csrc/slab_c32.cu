// Cluster-fused pass A instantiated for one storage type.
#define WSFFT_STORE float2
#define WSFFT_SLAB_NAME launch_slab_c32
#include "slab_launch.cuh"
