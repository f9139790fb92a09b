// int32 instantiation of the update launch sequences.
#include "launch.cuh"
namespace apsp {
APSP_INSTANTIATE(int32_t)
}
