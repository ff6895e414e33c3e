// Lane-group FP32 Dormand-Prince 5(4) integrator with the parameter records
// in registers, compiled at run time for one network's row layout.
//
// Model, lane mapping, gather buffer and step control are those of the
// shared-memory-record kernel (integrate_grp.cuh; GRiNS Sec. 2.1.1, Eq. 1
// and Eq. 2 written as products of w (p + u) / (1 + p), p = 2^t,
// t = n log2 x_src - n log2 T).  What differs:
//   * a lane keeps the records of its own edge positions in registers --
//     n, -n log2 T and 1/lambda as FP32 pairs, and the shared-memory address
//     of each position's source entry -- together with G', k and k/G of its
//     rows, loaded when it starts a solve.  The edge loop then issues one
//     shared load per edge (the source value) where the shared-record kernel
//     issues two, one of them 16 bytes wide;
//   * edges are taken two at a time with the packed FP32 pair instructions
//     (fma/add/mul .f32x2 of sm_100 and later), each pair component carrying
//     at most four factors (p <= 2^30) before its division;
//   * work is handed out one solve at a time from a set-major counter, so
//     no parameter-set slots are needed.
// The rows (GrpRowCt<r>: position offset and degree; kGrpCtRows) are
// compile-time constants generated for the network, and the stages of an
// attempt are written out, so every register array is indexed by constants
// and the gather buffer of each right-hand side is an immediate offset.
//
// FP64 instantiation (the plain FP64 GPU solver): the same body with double
// states and records; its edge term is exact rather than log-domain -- the
// gather buffer holds x, x^2 .. x^6 of every stage value and an edge forms
// p = x^n (1/T)^n with one multiply (n <= 6, Table 1; an edge with a larger
// n makes its solve non-finite), numerators and denominators divided once
// per eight factors.
#pragma once

#include "integrate_grp.cuh"

namespace grins {
#include "integrate_rr_layout.inc"
}  // namespace grins
