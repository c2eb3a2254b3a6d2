/*
 * sampler.c - FP64 CPU oracle of the candidate sampler: the paper draws the
 * N control sequences of every plan on the GPU (Sec. IV-D: i.i.d. samples of
 * the admissible controls, drawn with cuRAND); the serving path here draws
 * them as Gaussian perturbations of a warm-start nominal, with the
 * counter-based generator Philox4x64-10 (Salmon, Moraes, Dror, Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC'11) and the Box-Muller
 * transform (Box and Muller, 1958).
 *
 * TEST INFRASTRUCTURE.  Only the test suite may load it; it shares no code
 * with the CUDA sampler, which implements the same published definitions
 * separately.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

/* Philox4x64 round constants (Salmon et al. 2011, Table 2 and Sec. 3) */
#define PHILOX_M0 0xD2E7470EE14C6C93ull
#define PHILOX_M1 0xCA5A826395121157ull
#define PHILOX_W0 0x9E3779B97F4A7C15ull
#define PHILOX_W1 0xBB67AE8584CAA73Bull

static void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    unsigned __int128 p = (unsigned __int128)a * b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

/* ten rounds of the Philox S-P network, the key bumped by the Weyl
 * constants between rounds */
void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    uint64_t c[4], k0 = key[0], k1 = key[1];
    int r;
    memcpy(c, ctr, sizeof c);
    for (r = 0; r < 10; ++r) {
        uint64_t hi0, lo0, hi1, lo1, n[4];
        if (r > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        mulhilo64(PHILOX_M0, c[0], &hi0, &lo0);
        mulhilo64(PHILOX_M1, c[2], &hi1, &lo1);
        n[0] = hi1 ^ c[1] ^ k0;
        n[1] = lo1;
        n[2] = hi0 ^ c[3] ^ k1;
        n[3] = lo0;
        memcpy(c, n, sizeof c);
    }
    memcpy(out, c, sizeof c);
}

/* 23-bit uniform on (0, 1) from the high (bits 63..41) or low (bits 31..9)
 * half of a 64-bit Philox word */
static double unif23(uint64_t w, int low)
{
    uint64_t b = low ? (w >> 9) & 0x7FFFFFull : w >> 41;
    return ((double)b + 0.5) * (1.0 / 8388608.0);
}

/* Candidate controls ctrl[k][j] = nominal[k] + (sigma_rate n1, sigma_acc n2)
 * with (n1, n2) a Box-Muller pair of 23-bit uniforms.  One Philox call at
 * counter (j, kq, nonce, 0) serves the four steps k = 4 kq + s, s = 0..3: its
 * words (w0, w1) for s = 0 and 2, (w2, w3) for s = 1 and 3, their high
 * halves for s < 2 and their low halves for s >= 2.  Candidate 0 is the
 * nominal itself.  nominal[k] is the warm start prev[min(k + shift,
 * H_prev - 1)] (zero when H_prev = 0). */
void orc_sample(const float *prev, int H_prev, int shift, double sigma_rate, double sigma_acc,
                uint64_t key0, uint64_t key1, uint64_t nonce, int N, int H, double *out)
{
    const uint64_t key[2] = { key0, key1 };
    int j, k;
    for (k = 0; k < H; ++k) {
        double nom[2] = { 0.0, 0.0 };
        if (H_prev > 0) {
            int src = k + shift;
            if (src > H_prev - 1) src = H_prev - 1;
            nom[0] = prev[2 * src];
            nom[1] = prev[2 * src + 1];
        }
        for (j = 0; j < N; ++j) {
            double *o = out + ((size_t)k * N + j) * 2;
            if (j == 0) {
                o[0] = nom[0];
                o[1] = nom[1];
            } else {
                uint64_t ctr[4] = { (uint64_t)j, (uint64_t)(k / 4), nonce, 0 }, w[4];
                int s = k % 4, low = s >= 2;
                double u1, u2, r;
                orc_philox4x64_10(ctr, key, w);
                u1 = unif23((s & 1) ? w[2] : w[0], low);
                u2 = unif23((s & 1) ? w[3] : w[1], low);
                r = sqrt(-2.0 * log(u1));
                o[0] = nom[0] + sigma_rate * r * cos(2.0 * M_PI * u2);
                o[1] = nom[1] + sigma_acc * r * sin(2.0 * M_PI * u2);
            }
        }
    }
}
