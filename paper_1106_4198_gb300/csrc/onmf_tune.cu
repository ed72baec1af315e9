// onmf_autotune: picks the schedule of the mixed-precision online step for a
// shape by timing every candidate on a synthetic stream (CUDA events on the
// caller's stream): the h-solve kernel, which sets the frames per tile (mma
// 8, tcgen05 16, cluster 32), and for the mma kernel the frame ranges of the
// tcgen05 statistics (onmf_config.stats_ranges). An optional cache file of
// JSON lines keyed by the device name and the shape keeps the choice.
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "onmf.h"

namespace {

// Positive synthetic frames v = -log(u) + 1e-3 with u uniform from a
// counter hash (Wellons' "lowbias32" integer hash); only the timing of the
// kernels matters here, not the values.
__global__ void tune_fill(float *V, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        unsigned x = (unsigned)i * 2654435761u + 0x9e3779b9u;
        x ^= x >> 16;
        x *= 0x7feb352du;
        x ^= x >> 15;
        x *= 0x846ca68bu;
        x ^= x >> 16;
        const float u = (float)(x >> 8) * (1.0f / 16777216.0f) + 1e-7f;
        V[i] = -logf(u) + 1e-3f;
    }
}

struct Key {
    std::string device;
    int F, K, beta, n_inner;
};

bool same(const Key &a, const Key &b) {
    return a.device == b.device && a.F == b.F && a.K == b.K && a.beta == b.beta &&
           a.n_inner == b.n_inner;
}

// Statistics schedules tried with the mma h-solve (0: automatic).
constexpr int kRangeCands[5] = {0, 2, 4, 8, 16};

struct Choice {
    int hsolve = -1, ranges = 0;
    double us[4] = {-1.0, -1.0, -1.0, -1.0};      // best per kernel
    double rus[5] = {-1.0, -1.0, -1.0, -1.0, -1.0};  // mma kernel per range candidate
};

int tile_frames(int h) { return h == ONMF_HSOLVE_MMA ? 8 : h == ONMF_HSOLVE_TC ? 16 : 32; }

// One cache line: {"device": "...", "F": 513, "K": 100, "beta": 1000,
// "n_inner": 10, "hsolve": 1, "tile_frames": 8, "stats_ranges": 0,
// "us_per_minibatch": [a, b, c, d], "stats_ranges_us": [e, f, g, h, i]}
bool parse(const char *line, Key &k, Choice &c) {
    const char *d = strstr(line, "\"device\": \"");
    if (!d) return false;
    d += strlen("\"device\": \"");
    const char *e = strchr(d, '"');
    if (!e) return false;
    k.device.assign(d, e - d);
    int tf = 0;
    return sscanf(e + 1,
                  ", \"F\": %d, \"K\": %d, \"beta\": %d, \"n_inner\": %d, \"hsolve\": %d, "
                  "\"tile_frames\": %d, \"stats_ranges\": %d, "
                  "\"us_per_minibatch\": [%lf, %lf, %lf, %lf], "
                  "\"stats_ranges_us\": [%lf, %lf, %lf, %lf, %lf]}",
                  &k.F, &k.K, &k.beta, &k.n_inner, &c.hsolve, &tf, &c.ranges, &c.us[0], &c.us[1],
                  &c.us[2], &c.us[3], &c.rus[0], &c.rus[1], &c.rus[2], &c.rus[3],
                  &c.rus[4]) == 16;
}

}  // namespace

extern "C" onmf_status onmf_autotune(const onmf_config *cfg, void *stream, const char *cache_path,
                                     int32_t *hsolve_out, int32_t *stats_ranges_out,
                                     double *us_out, double *ranges_us_out,
                                     int32_t *from_cache) {
    if (!cfg || !hsolve_out) return ONMF_EINVAL;
    Choice best;
    auto give = [&](const Choice &c) {
        *hsolve_out = c.hsolve;
        if (stats_ranges_out) *stats_ranges_out = c.ranges;
        if (us_out) memcpy(us_out, c.us, sizeof c.us);
        if (ranges_us_out) memcpy(ranges_us_out, c.rus, sizeof c.rus);
    };
    if (from_cache) *from_cache = 0;
    if (cfg->precision != ONMF_MIXED) {
        best.hsolve = ONMF_HSOLVE_AUTO;  // the FP32 path has one h-solve
        give(best);
        return ONMF_OK;
    }
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
        return ONMF_ECUDA;
    const Key key{prop.name, cfg->F, cfg->K, cfg->beta, cfg->n_inner};
    if (cache_path) {
        if (FILE *f = fopen(cache_path, "r")) {
            char line[1024];
            Choice found;
            while (fgets(line, sizeof line, f)) {
                Key k;
                Choice c;
                if (parse(line, k, c) && same(k, key)) found = c;
            }
            fclose(f);
            if (found.hsolve > 0) {
                give(found);
                if (from_cache) *from_cache = 1;
                return ONMF_OK;
            }
        }
    }
    cudaStream_t q = reinterpret_cast<cudaStream_t>(stream);
    const int warm = 3, timed = 20;
    const long long frames = (long long)(warm + timed) * cfg->beta;
    float *V = nullptr;
    if (cudaMalloc((void **)&V, (size_t)frames * cfg->F * 4) != cudaSuccess) return ONMF_ENOMEM;
    tune_fill<<<1024, 256, 0, q>>>(V, frames * cfg->F);
    std::vector<float> W0((size_t)cfg->F * cfg->K);
    for (size_t i = 0; i < W0.size(); ++i) W0[i] = 1.0f / cfg->F * (1.0f + 0.5f * (float)((i * 7919) % 13) / 13.f);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best_us = -1.0;
    onmf_status rc = ONMF_OK, dropped = ONMF_OK;
    for (int h = ONMF_HSOLVE_MMA; h <= ONMF_HSOLVE_CLUSTER && rc == ONMF_OK; ++h) {
        const int nr = h == ONMF_HSOLVE_MMA ? 5 : 1;
        for (int ri = 0; ri < nr && rc == ONMF_OK; ++ri) {
            onmf_config c = *cfg;
            c.hsolve = h;
            c.stats_ranges = kRangeCands[ri];
            onmf_state *s = nullptr;
            if (onmf_init(&c, W0.data(), 0, stream, &s) != ONMF_OK) break;  // not for this shape
            rc = onmf_push_frames(s, V, c.F, (long long)warm * c.beta, nullptr, 0);
            if (rc == ONMF_OK) rc = onmf_synchronize(s);
            if (rc == ONMF_OK) {
                cudaEventRecord(e0, q);
                rc = onmf_push_frames(s, V + (size_t)warm * c.beta * c.F, c.F,
                                      (long long)timed * c.beta, nullptr, 0);
                cudaEventRecord(e1, q);
            }
            if (rc == ONMF_OK) rc = onmf_synchronize(s);
            onmf_destroy(s);
            if (rc != ONMF_OK) {
                // A kernel that reported an error through its status word (a
                // wait that timed out, a launch shape its entry check refused)
                // leaves the context usable: drop that candidate and go on. A
                // CUDA error that the context keeps ends the tuning.
                if (cudaStreamSynchronize(q) != cudaSuccess || cudaPeekAtLastError() != cudaSuccess)
                    break;
                dropped = rc;
                rc = ONMF_OK;
                continue;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            const double us = 1e3 * ms / timed;
            if (h == ONMF_HSOLVE_MMA) best.rus[ri] = us;
            if (best.us[h] < 0 || us < best.us[h]) best.us[h] = us;
            if (best_us < 0 || us < best_us) {
                best_us = us;
                best.hsolve = h;
                best.ranges = c.stats_ranges;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(V);
    if (rc != ONMF_OK) return rc;
    if (best.hsolve < 0) return dropped != ONMF_OK ? dropped : ONMF_EINVAL;
    give(best);
    if (cache_path) {
        if (FILE *f = fopen(cache_path, "a")) {
            fprintf(f,
                    "{\"device\": \"%s\", \"F\": %d, \"K\": %d, \"beta\": %d, \"n_inner\": %d, "
                    "\"hsolve\": %d, \"tile_frames\": %d, \"stats_ranges\": %d, "
                    "\"us_per_minibatch\": [%.3f, %.3f, %.3f, %.3f], "
                    "\"stats_ranges_us\": [%.3f, %.3f, %.3f, %.3f, %.3f]}\n",
                    key.device.c_str(), key.F, key.K, key.beta, key.n_inner, best.hsolve,
                    tile_frames(best.hsolve), best.ranges, best.us[0], best.us[1], best.us[2],
                    best.us[3], best.rus[0], best.rus[1], best.rus[2], best.rus[3], best.rus[4]);
            fclose(f);
        }
    }
    return ONMF_OK;
}
