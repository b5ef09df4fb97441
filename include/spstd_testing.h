/*
 * spstd_testing.h -- test hooks of the SPSTD library (include/spstd.h).
 *
 * Not part of the solver API: these entry points exist so that tests can drive
 * failure paths that a correct run never takes.  They are exported by
 * libspstd.so like the rest and follow the same conventions.
 */
#ifndef SPSTD_TESTING_H
#define SPSTD_TESTING_H

#include "spstd.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Test hook for the failure path of the bounded device waits.  With the
 * fused x-y pass active: makes its next launch skip one y tile of its first
 * plane, so that the x tiles of that plane wait in vain until their bounded
 * waits run out (about a second).  Otherwise, on a context whose x axis runs
 * the default pipelined (TMA) pass: makes the next x pass (or fused
 * reduce-add x-y pass) leave its first tile unloaded, so that the wait on
 * that tile's barrier runs out (about two seconds);
 * the block then waits for the loads it still has in flight and returns.
 * Either way the blocks return early with the device status word set, the
 * next synchronising call reports SPSTD_ETIMEOUT and clears the status;
 * psi_R and psi_I are left partly updated, and the context stays usable (set
 * a state and step again).  SPSTD_EUNSUPPORTED when the context has neither
 * pass. */
spstd_status spstd_inject_wait_timeout(spstd_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif
