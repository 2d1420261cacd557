// Instantiation: keys uint64_t, values: uint64_t.
#define DTS_K uint64_t
#define DTS_HV true
#define DTS_NAME u64kv
#include "dtsort_inst.cuh"
