// Cluster-fused pass A instantiated for one storage type.
#define WSFFT_STORE __nv_bfloat162
#define WSFFT_SLAB_NAME launch_slab_c16bf
#include "slab_launch.cuh"
