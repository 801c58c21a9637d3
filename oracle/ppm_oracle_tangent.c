/*
 * ppm_oracle_tangent.c -- forward-mode (tangent) build of the FP64 oracle.
 *
 * TEST INFRASTRUCTURE ONLY, like ppm_oracle.c: used by the test-suite to
 * obtain exact directional derivatives of the oracle's log-likelihood.
 *
 * The oracle source is compiled a second time with real = double complex;
 * the header of ppm_oracle.c describes how a parameter is seeded and why the
 * imaginary part of the result is h times the derivative along the seed.
 * Only orc_loglike_full is called from this build.
 */
#define ORC_CSTEP 1
#include "ppm_oracle.c"
