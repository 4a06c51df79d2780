// Mixed-precision line searches: the contractions run on the BF16 tensor
// cores (tcgen05, TMEM accumulators, TMA-fed shared memory) as 3-term split
// products with FP32 accumulation; the state stays in float64.
#pragma once
#include "omm_internal.cuh"

namespace omm {

struct MixedState;

MixedState* mixed_create(cudaStream_t st, int m, int n, const double* HS, const double* P);
void mixed_update_H(MixedState* ms, cudaStream_t st, const double* HS);
void mixed_destroy(MixedState* ms);
void mixed_iterate(MixedState* ms, cudaStream_t st, Scalars* sc, double* C, double* Dir, double* G,
                   double* Gold, double* PG, double* Y4, double* SWHW, double* Proj, double* part,
                   double* part2, const double* HS, const double* P, bool precond);

}  // namespace omm
