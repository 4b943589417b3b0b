// gs_loop.cuh -- the loop kernel of the GridShift hot path (Kumar et al.,
// arXiv 2206.02200, Sec. 2.1 and Algorithm 1): one cooperative launch for
// everything between the first binning pass and the labels (for runs of
// 2^22 points or more, binning's second pass and the label writes are
// launches of their own around it):
//   binning, second pass: exact cell sums through a counting sort of the
//            points by cell (step i)
//   level 0: the initial cells and their table
//   per update step t:
//     update   steps ii-iv: Eq. 1-2 over the 3^d neighbours in the parallel
//              form (Eq. 6), centroid, new key, and the neighbour test of
//              step v; the count-weighted centroid merged (Eq. 3-4) into the
//              slot of the new key
//     compact  the next level's cells and sums
//   then the forest of merges (the union of resident sets of Eq. 4) is
//   resolved by pointer jumping, the final cells are numbered by ascending
//   key, and every point gets its label.
// Phases are separated by a software grid barrier whose waits are bounded in
// time.  Included by gs_loop64.cu (exact sums rounded once to float64) and
// gs_loop32.cu (the float32 mixed-precision variant), which instantiate it.
//
// The code is in five parts, each including the one before: gs_loop_base.cuh
// (barrier, clock, helpers), gs_loop_fp64.cuh (the exact path's phases),
// gs_loop_fp32.cuh (the float32 path's phases), gs_loop_tail.cuh (the
// one-block tails) and gs_loop_kernel.cuh (the kernels and launch helpers).
#pragma once

#include "gs_loop_kernel.cuh"
