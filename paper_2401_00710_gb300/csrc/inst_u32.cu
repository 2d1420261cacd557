// Instantiation: keys uint32_t, values: none.
#define DTS_K uint32_t
#define DTS_HV false
#define DTS_NAME u32
#include "dtsort_inst.cuh"
