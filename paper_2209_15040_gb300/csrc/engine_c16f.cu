// Persistent engine instantiated for storage type __half2.
#define WSFFT_STORE __half2
#define WSFFT_ENGINE_NAME launch_engine_c16f
#define WSFFT_PERSIST_NAME launch_persist_c16f
#define WSFFT_WPP_NAME launch_wpp_c16f
#define WSFFT_WPS_NAME launch_wps_c16f
#include "engine_launch.cuh"
