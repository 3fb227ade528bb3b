// FP64 kernels (ALU-bound on GB300).  Variants as in the FP32 unit:
//   1  v1  64  5  no   2
//   2  v2  64  5  no   2
//   3  v2  64  4  yes  3
//   4  v3  64  5  no   2   (tensor-map TMA)
//   5  v3  64  4  yes  3   (tensor-map TMA)
#include "dbm.h"
#define DBM_REAL double
#define DBM_VARIANTS(X) X(1, 1, 64, 5, false, 2) X(2, 2, 64, 5, false, 2) X(3, 2, 64, 4, true, 3) \
    X(4, 3, 64, 5, false, 2) X(5, 3, 64, 4, true, 3)
#define DBM_DEFAULT_VARIANT 2
#define DBM_FALLBACK_VARIANT 2
#define DBM_BATCH_CONST_SLOTS DBM_BATCH_CONST_FP64  // batch constant table entries (304 B each)
#include "dbm_launch_impl.cuh"
