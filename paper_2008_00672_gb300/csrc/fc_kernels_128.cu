// The generic kernels of fc_kernels.cu compiled for 128-thread CTAs, four resident per SM,
// for plans whose transforms all fit them (batch 2 of at most 1024 points) and whose
// shared memory fits four times per SM. Exported as fc_gen_kernels_128().
#define FC_THREADS 128
#define FC_GEN_MIN_BLOCKS 4
#include "fc_kernels.cu"
