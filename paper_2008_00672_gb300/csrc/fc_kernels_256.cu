// The generic kernels of fc_kernels.cu compiled for 256-thread CTAs, two resident per SM.
// Plans whose transforms all fit (batch 2 of at most 2048 points) and whose shared memory
// fits twice per SM run on this set: with two CTAs per SM, one CTA's barrier waits overlap
// the other's work. The set is exported as fc_gen_kernels_256().
#define FC_THREADS 256
#define FC_GEN_MIN_BLOCKS 2
#include "fc_kernels.cu"
