// gint_dm.cuh -- the tensor-core density-matrix build used by the dense-step context.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

// Device bytes of the work buffer gint_dm_tc needs for an n x n matrix and nocc states (the packed
// float16 hi / lo operands and two scale words).
size_t gint_dm_tc_bytes(int n, int nocc);

// D (n x n float64, device) = Re(psi diag(f) psi^dagger) in the float16 three-term split on the
// tensor cores; psi: nocc rows of n complex128 (device); f: nocc occupations (device, any sign);
// work: gint_dm_tc_bytes(n, nocc) device bytes; status: device word, bit 1 set when a bounded wait
// gave up.  Asynchronous on st.
int gint_dm_tc(int n, int nocc, const double *psi, const double *f, double *D, void *work, unsigned *status,
               cudaStream_t st);
