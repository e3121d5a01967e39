// Persistent engine instantiated for storage type __nv_bfloat162.
#define WSFFT_STORE __nv_bfloat162
#define WSFFT_ENGINE_NAME launch_engine_c16bf
#define WSFFT_PERSIST_NAME launch_persist_c16bf
#define WSFFT_WPP_NAME launch_wpp_c16bf
#define WSFFT_WPS_NAME launch_wps_c16bf
#include "engine_launch.cuh"
