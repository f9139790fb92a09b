// Training and batched inference kernels of the warm/cold cost model
// (see mlp.cuh for the network and the parameter layout).
#include "apsp.h"
#include "mlp.cuh"
