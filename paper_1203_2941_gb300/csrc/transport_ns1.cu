// Transport kernel variants for one density species (packed width 1); the kernels
// and their launchers are in transport.cu.
#define RT_TRANSPORT_NS 1
#include "transport.cu"
