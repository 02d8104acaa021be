// Transport kernel variants for two density species (packed width 2); the kernels
// and their launchers are in transport.cu.
#define RT_TRANSPORT_NS 2
#include "transport.cu"
