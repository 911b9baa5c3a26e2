/*
 * scint_testing.h -- inspection entry points of libscint.so.
 *
 * They expose intermediate quantities of the hot path so that tests can check
 * them one by one against an independent reference.  Same conventions as
 * scint.h (device pointers, stream ordering, status codes, scint_last_error).
 */
#ifndef SCINT_TESTING_H
#define SCINT_TESTING_H

#include <stddef.h>
#include <stdint.h>

#include "scint.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Raw Philox4x32-10 words of the screen's noise stream (Sect. 3.1: the random
 * complex numbers behind F_phi).  Bin (ky, kx) uses counter
 * (kx, ky, screen_id, 0) and key (seed low 32 bits, seed high 32 bits).
 *   words  device, N*N*4 uint32, row-major by (ky, kx), 4 words per bin.
 */
int scint_noise_words(const scint_params* p, uint32_t* words, void* stream);

/*
 * The shaped random spectrum F_phi of Eq. densite, exactly as the synthesis
 * generates it: F = sqrt(L^2 S_phi(q)) (g_re + i g_im)/sqrt(2), F(0) = 0.
 *   F  device, N*N complex128 (interleaved re, im), row-major by (ky, kx),
 *      FFT frequency order.
 */
int scint_noise_spectrum(const scint_params* p, double* F, void* stream);

/*
 * The library's line FFT applied to n_lines contiguous lines of length n:
 * out_k = sum_j in_j exp(dir 2 pi i j k / n), unnormalised, dir = -1 or +1.
 *   data  device, n_lines*n complex64 (FP32) or complex128 (FP64), in place.
 */
int scint_fft_lines32(int n, int dir, float* data, int n_lines, void* stream);
int scint_fft_lines64(int n, int dir, double* data, int n_lines, void* stream);

/*
 * The propagation passes' fixed-point phase (exact mod 2 pi reduction, Sect. 3.2.4
 * phi_lambda = phi lambda_ref / lambda): P_i = round(phi_i 2^32 / 2 pi) as the row
 * passes compute it: one FP64 product, rounded to the nearest integer (clamped to the
 * int64 range).
 *   phi  device, n doubles;  P  device, n int64.  n >= 0.
 */
int scint_phase_fixed(const double* phi, int64_t* P, int64_t n, void* stream);

/*
 * Failure injection for the persistent batch kernel (scint_batch_mode 1), on the
 * host: the next launches count screen `withhold` (its index in the batch) as
 * having one more row item than it has, so the waits for its row work cannot
 * succeed, and give up each wait after `wait_limit` counter reads (about 0.2 us
 * apart; <= 0 restores the default of about 2 s).  withhold < 0 turns it off.
 * The launch then ends early with SCINT_ETIMEOUT in its status word
 * (scint_batch_status) and incomplete outputs; nothing faults or hangs.
 */
void scint_testing_persist(int withhold, int wait_limit);

#ifdef __cplusplus
}
#endif

#endif /* SCINT_TESTING_H */
