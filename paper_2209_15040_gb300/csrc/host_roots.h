// Host-side roots of unity and stage-twiddle tables, shared by the plan
// builder and the allocation-free entry point (one generator for both).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace wsfft {

// exp(-2*pi*i*m/n): the angle is reduced to the first octant by the
// eight-fold symmetry of the unit circle, evaluated in long double, then
// rounded to float (twiddles computed in higher precision and rounded once).
float2 host_root(int64_t m, int64_t n);

// Stage-twiddle table of the (N, E) register schedule (fft_core.cuh: stage
// s >= 1 reads w_{Ns*R}^{r*k} at sched_tw_offset(s) + (r-1)*Ns + k), plus one
// zero pad entry.  Writes at most `cap` entries to dst and returns how many
// it wrote, or -1 if the table does not fit.
int fill_stage_table(float2 *dst, int cap, int N, int E);

}  // namespace wsfft
