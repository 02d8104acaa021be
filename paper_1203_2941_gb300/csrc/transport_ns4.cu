// Transport kernel variants for three or four density species (packed width 4); the kernels
// and their launchers are in transport.cu.
#define RT_TRANSPORT_NS 4
#include "transport.cu"
