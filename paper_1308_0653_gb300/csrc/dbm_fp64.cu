// FP64 kernels: 64 radial sites per CTA, 5-deep row ring (92 KB shared).
#define DBM_REAL double
#define DBM_W 64
#define DBM_NSTAGE 5
#include "dbm_launch_impl.cuh"
