// The particle-by-particle move kernel for CTAs of 128 threads, mixed path
// (qmc_move_impl.cuh).
#define QMCGB_MOVE_NT 128
#define QMCGB_MOVE_NS nt128
#define QMCGB_MOVE_ELEM 4
#include "qmc_move_impl.cuh"
