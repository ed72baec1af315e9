/* C client of libonmf (include/onmf.h): one online pass over host frames of
 * a small synthetic spectrogram in FP32 and in mixed precision, then a
 * projection of the same frames, all through the plain C ABI.
 * Exits 0 when every call succeeds and the results are finite and
 * nonnegative; prints one line per check. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "onmf.h"

#define F 65
#define K 6
#define N 200

static unsigned rng_state = 12345u;
static float urand(void) { /* xorshift32 */
    rng_state ^= rng_state << 13;
    rng_state ^= rng_state >> 17;
    rng_state ^= rng_state << 5;
    return ((rng_state >> 8) + 0.5f) * (1.0f / 16777216.0f);
}

static int check(const char *what, onmf_status st) {
    printf("%-28s %s\n", what, onmf_status_string(st));
    if (st != ONMF_OK) {
        printf("  detail: %s\n", onmf_last_error_message());
        return 1;
    }
    return 0;
}

static int all_finite_nonneg(const float *x, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!(x[i] >= 0.f) || isinf(x[i])) return 0;
    return 1;
}

int main(void) {
    static float V[N * F], W0[F * K], W[F * K], H[N * K];
    int bad = 0;
    for (size_t i = 0; i < (size_t)N * F; ++i) V[i] = -logf(urand()) + 1e-3f;
    for (int k = 0; k < K; ++k) { /* column-major F x K, unit column sums */
        float s = 0.f;
        for (int f = 0; f < F; ++f) s += (W0[f + k * F] = urand() + 0.1f);
        for (int f = 0; f < F; ++f) W0[f + k * F] /= s;
    }
    if (onmf_abi_version() != ONMF_ABI_VERSION) {
        printf("ABI version mismatch\n");
        return 1;
    }
    for (int prec = ONMF_FP32; prec <= ONMF_MIXED; ++prec) {
        onmf_config cfg;
        onmf_state *s = NULL;
        onmf_config_default(&cfg, F, K);
        cfg.beta = 32;
        cfg.n_inner = 5;
        cfg.precision = prec;
        bad |= check(prec ? "init (mixed)" : "init (fp32)", onmf_init(&cfg, W0, 0, NULL, &s));
        if (!s) return 1;
        bad |= check("push_frames (host)", onmf_push_frames(s, V, F, N, H, K));
        bad |= check("flush", onmf_flush(s));
        bad |= check("get_W", onmf_get_W(s, W, 0));
        int64_t t = 0;
        double loss = 0.0;
        bad |= check("get_stats", onmf_get_stats(s, NULL, NULL, &t, &loss));
        double obj = 0.0;
        bad |= check("project (host)", onmf_project(s, V, F, N, H, K, -1, &obj));
        printf("  frames %lld, loss/frame %.4f, projected objective/frame %.4f\n", (long long)t,
               loss / (double)t, obj / N);
        bad |= !(t == N && isfinite(loss) && loss > 0.0 && isfinite(obj) && obj > 0.0);
        bad |= !all_finite_nonneg(W, (size_t)F * K) || !all_finite_nonneg(H, (size_t)N * K);
        onmf_destroy(s);
    }
    printf("%s\n", bad ? "FAILED" : "OK");
    return bad;
}
