/*
 * lbvdw_selftest.h -- self-test entry points of the lbvdw library (not part of the
 * lattice Boltzmann step).  lb_selftest_log exposes the two logarithms the
 * chemical-potential stage uses on GB300 so that tests can compare them with CUDA's
 * double-precision log on the same device (lb_selftest_recip does the same for its
 * double-float reciprocal):
 *   - the table-driven FP64 logarithm of the LB_FP32_MIXED path;
 *   - the double-float logarithm of the LB_FP32_DFMU path.
 * The chemical potential that needs these logarithms is Eq. discreteChemicalPotential
 * of Ridl & Wagner (arXiv:1805.07251), mu^c = kT ln(rho^c/eta) + ...
 */
#ifndef LBVDW_SELFTEST_H
#define LBVDW_SELFTEST_H

#include "lbvdw.h"

#ifdef __cplusplus
extern "C" {
#endif

/* For n host values x[k] > 0 (normal, finite) compute on device `device`:
 *   out_tbl[k] = table-driven FP64 log(x[k]),
 *   out_df[k]  = double-float log of x[k] (x first rounded to a double-float pair),
 *                returned as hi + lo in double,
 *   out_ref[k] = CUDA's double-precision log(x[k]).
 * All arrays are host arrays of n doubles owned by the caller.  Allocates and frees
 * its own device scratch; synchronous.  Errors: LB_E_INVALID (NULL pointer, n < 1),
 * LB_E_NOMEM, LB_E_CUDA. */
lb_status lb_selftest_log(int32_t device, const double *x, int64_t n, double *out_tbl, double *out_df,
                          double *out_ref);

/* For n host values x[k] > 0 (normal, finite, x[k] and 1/x[k] within the float range)
 * compute on device `device` out_df[k] = 1/x[k] by the double-float reciprocal of the
 * LB_FP32_DFMU chemical potential (the 1/eta = 1/(1 - sum_c b^c rho^c) of Eq.
 * discreteChemicalPotential), x first rounded to a double-float pair and the result
 * returned as hi + lo in double.  Host arrays of n doubles owned by the caller; allocates
 * and frees its own device scratch; synchronous.  Errors: LB_E_INVALID (NULL pointer,
 * n < 1), LB_E_NOMEM, LB_E_CUDA. */
lb_status lb_selftest_recip(int32_t device, const double *x, int64_t n, double *out_df);

/* The bounded wait that the streaming-strip kernel (LB_KERNEL_STRIPS) applies to its
 * bulk-copy barriers, run on one CTA of 64 threads on device `device` against an mbarrier
 * that completes (arrive != 0: thread 0 arrives) or that nothing ever completes
 * (arrive == 0).  Every thread polls at most `polls` times; *flag receives the error word:
 * 0 when the barrier completed, 2 (the timeout bit, reported as LB_E_TIMEOUT by the step
 * calls) when the polls ran out.  No fault, no hang: the wait ends either way.
 * Synchronous.  Errors: LB_E_INVALID (NULL flag, polls < 1), LB_E_NOMEM, LB_E_CUDA. */
lb_status lb_selftest_wait(int32_t device, uint32_t polls, int32_t arrive, uint32_t *flag);

/* The bounded wait of a chained step (lb_step with two or more steps, LB_FP32_DFMU /
 * LB_FP32, two components, D2Q9) on a neighbouring tile's completion flag, run by one
 * thread on device `device` against a flag that already holds the awaited step (set != 0)
 * or never will (set == 0: it holds the step before, and nothing writes it).  The wait
 * gives up after wait_ns nanoseconds of GPU time; *flag receives the error word: 0 when the
 * flag was reached, 4 (the stall bit, reported as LB_E_TIMEOUT by lb_step) when the bound
 * ran out.  No fault, no hang: the wait ends either way.  Synchronous.  Errors:
 * LB_E_INVALID (NULL flag, wait_ns < 1 or > 10^10), LB_E_NOMEM, LB_E_CUDA. */
lb_status lb_selftest_flag_wait(int32_t device, uint64_t wait_ns, int32_t set, uint32_t *flag);

#ifdef __cplusplus
}
#endif
#endif /* LBVDW_SELFTEST_H */
