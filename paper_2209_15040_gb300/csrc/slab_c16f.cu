// Cluster-fused pass A instantiated for one storage type.
#define WSFFT_STORE __half2
#define WSFFT_SLAB_NAME launch_slab_c16f
#include "slab_launch.cuh"
