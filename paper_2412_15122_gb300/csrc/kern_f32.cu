// float instantiation of the update launch sequences.
#include "launch.cuh"
namespace apsp {
APSP_INSTANTIATE(float)
}
