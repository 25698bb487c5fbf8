// autotune.cu -- launch-shape selection for the wavelet predictors.
//
// The best shape (threads per CTA x visibilities per thread) depends on the
// tree (depth J sets the per-thread stack, node count the work per
// visibility) and on the form. The first call for a new key times every
// shape that fits on one sample of the caller's own visibilities (float64
// forms: two waves of the resident CTAs of the shape that holds the most,
// at least 131 072; mixed forms: up to 2 Mi; never more than the batch;
// written into the caller's output buffer, which the real launch then
// overwrites), a warm-up and the best of two timed launches each, and
// remembers the fastest. Keys are (device, form,
// sum, J, log2 of the node count, log2 of the leaf count).
//
// Tuning synchronises the caller's stream once. It is skipped, in favour of
// the default shape, when WT_AUTOTUNE=0 is set or when the stream is being
// captured into a CUDA graph. With WT_TUNE_CACHE=<path> the results are also
// read from and appended to a text file, one "key variant" pair per line.
// WT_AUTOTUNE_VERBOSE=1 prints every timed shape to stderr.
// WT_WAVELET_VARIANT=<k> pins shape k (see kVariants in wavelet.cu) when it
// fits, overriding both the cache and the tuning.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>

#include "wt_internal.cuh"

namespace wt {
namespace {

std::mutex g_mu;
std::map<std::string, int> g_cache;
bool g_file_loaded = false;

int ilog2(int64_t x)
{
    int r = 0;
    while (x > 1) {
        x >>= 1;
        ++r;
    }
    return r;
}

bool tuning_enabled()
{
    const char* e = getenv("WT_AUTOTUNE");
    return !(e && strcmp(e, "0") == 0);
}

bool verbose()
{
    const char* e = getenv("WT_AUTOTUNE_VERBOSE");
    return e && strcmp(e, "1") == 0;
}

void load_file_locked()
{
    if (g_file_loaded) return;
    g_file_loaded = true;
    const char* path = getenv("WT_TUNE_CACHE");
    if (!path) return;
    FILE* f = fopen(path, "r");
    if (!f) return;
    char key[256];
    int v;
    while (fscanf(f, "%255s %d", key, &v) == 2)
        if (v >= 0 && v < kNumWaveletVariants) g_cache[key] = v;
    fclose(f);
}

void append_file(const std::string& key, int v)
{
    const char* path = getenv("WT_TUNE_CACHE");
    if (!path) return;
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d\n", key.c_str(), v);
    fclose(f);
}

}  // namespace

// Two full waves of a variant's resident CTAs (as many as fit an SM by
// shared memory and threads; registers may admit fewer, which only adds
// waves), so that small-CTA shapes are measured at the occupancy they reach
// on a large batch, not on a sample that leaves SMs idle; at least 131072,
// at most the whole batch.
static int64_t sample_size(int v, const WaveletJob& jb)
{
    int nt = 0, vpt = 0;
    wavelet_variant_shape(v, &nt, &vpt);
    const size_t smem = wavelet_variant_smem(v, jb.mode, jb.which, jb.J) + 1024;   // + per-CTA reserve
    int64_t per_sm = static_cast<int64_t>((228 * 1024) / smem);
    if (per_sm > 2048 / nt) per_sm = 2048 / nt;
    if (per_sm > 32) per_sm = 32;
    if (per_sm < 1) per_sm = 1;
    int64_t n = 2 * static_cast<int64_t>(num_sms()) * per_sm * nt * vpt;
    if (n < 131072) n = 131072;
    return n < jb.n_vis ? n : jb.n_vis;
}

int choose_wavelet_variant(wt_tree t, const WaveletJob& jb, cudaStream_t s)
{
    const int fallback = default_wavelet_variant(jb.mode, jb.which, jb.J);
    const char* pin = getenv("WT_WAVELET_VARIANT");
    if (pin && *pin) {
        const int v = atoi(pin);
        if (wavelet_variant_fits(v, jb.mode, jb.which, jb.J)) return v;
    }
    if (!tuning_enabled()) return fallback;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();
        return fallback;
    }
    if (cs != cudaStreamCaptureStatusNone) return fallback;
    if (tree_sync_header(t) != WT_OK) return fallback;
    int dev = 0;
    cudaGetDevice(&dev);
    char kb[256];
    snprintf(kb, sizeof(kb), "wavelet:dev%d:mode%d:sum%d:J%d:T%d:L%d", dev, jb.mode, jb.which, jb.J,
             ilog2(t->host_hdr->n_nodes), ilog2(t->host_hdr->n_leaves));
    const std::string key(kb);
    {
        std::lock_guard<std::mutex> lk(g_mu);
        load_file_locked();
        auto it = g_cache.find(key);
        if (it != g_cache.end()) return it->second;
    }
    WaveletJob sample = jb;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        return fallback;
    }
    int best = fallback;
    float best_ms = 1e30f;
    // one sample for every shape: the largest two-wave size among them, so
    // that all are timed on the same visibilities with the GPU full
    int64_t common = 0;
    for (int v = 0; v < kNumWaveletVariants; ++v)
        if (wavelet_variant_fits(v, jb.mode, jb.which, jb.J)) {
            const int64_t n = sample_size(v, jb);
            if (n > common) common = n;
        }
    // the float32 mixed forms are fast enough to time on up to 2 Mi
    // visibilities: the shapes' last waves differ with the batch size, so
    // the closer the sample is to the real batch, the better the choice
    if (jb.mode == WT_MIXED || jb.mode == WT_MIXED_FAST) {
        const int64_t cap = int64_t(1) << 21;
        common = jb.n_vis < cap ? jb.n_vis : (common > cap ? common : cap);
    }
    sample.n_vis = common;
    for (int v = 0; v < kNumWaveletVariants; ++v) {
        if (!wavelet_variant_fits(v, jb.mode, jb.which, jb.J)) continue;
        if (launch_wavelet(sample, v, s) != WT_OK) continue;   // warm-up
        float ms = 1e30f;
        bool ok = true;
        for (int rep = 0; rep < 2 && ok; ++rep) {
            cudaEventRecord(e0, s);
            ok = launch_wavelet(sample, v, s) == WT_OK;
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess || !ok) {
                cudaGetLastError();
                ok = false;
                break;
            }
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            if (t < ms) ms = t;
        }
        if (!ok) continue;
        const float per_vis = ms / static_cast<float>(sample.n_vis);
        if (verbose()) {
            int nt = 0, vpt = 0;
            wavelet_variant_shape(v, &nt, &vpt);
            fprintf(stderr, "[wt autotune] %s variant %d (%d threads x %d vis): %.4f ms for %lld vis\n", key.c_str(), v,
                    nt, vpt, ms, static_cast<long long>(sample.n_vis));
        }
        if (per_vis < best_ms) {
            best_ms = per_vis;
            best = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_cache[key] = best;
    }
    append_file(key, best);
    return best;
}

}  // namespace wt
