// The particle-by-particle move kernel for CTAs of 160 threads, FP64 path
// (qmc_move_impl.cuh).
#define QMCGB_MOVE_NT 160
#define QMCGB_MOVE_NS nt160
#define QMCGB_MOVE_ELEM 8
#include "qmc_move_impl.cuh"
