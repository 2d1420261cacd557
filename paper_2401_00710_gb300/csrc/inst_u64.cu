// Instantiation: keys uint64_t, values: none.
#define DTS_K uint64_t
#define DTS_HV false
#define DTS_NAME u64
#include "dtsort_inst.cuh"
