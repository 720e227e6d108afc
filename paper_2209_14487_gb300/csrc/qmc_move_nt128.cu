// The particle-by-particle move kernel for CTAs of 128 threads (qmc_move_impl.cuh).
#define QMCGB_MOVE_NT 128
#define QMCGB_MOVE_NS nt128
#include "qmc_move_impl.cuh"
