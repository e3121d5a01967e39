// Persistent engine instantiated for storage type float2.
#define WSFFT_STORE float2
#define WSFFT_ENGINE_NAME launch_engine_c32
#define WSFFT_PERSIST_NAME launch_persist_c32
#define WSFFT_WPP_NAME launch_wpp_c32
#define WSFFT_WPS_NAME launch_wps_c32
#include "engine_launch.cuh"
