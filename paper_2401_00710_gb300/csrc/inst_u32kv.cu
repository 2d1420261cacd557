// Instantiation: keys uint32_t, values: uint32_t.
#define DTS_K uint32_t
#define DTS_HV true
#define DTS_NAME u32kv
#include "dtsort_inst.cuh"
