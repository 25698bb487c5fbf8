// autotune.cu -- launch-shape selection for the wavelet predictors.
//
// The best shape (threads per CTA x visibilities per thread) depends on the
// tree (depth J sets the per-thread stack, node count the work per
// visibility) and on the form. The first call for a new key times every
// shape that fits on a sample of the caller's own visibilities (two waves
// of the shape's resident CTAs, at least 131 072 and at most all of them,
// written into the caller's output buffer, which the real launch then
// overwrites) and remembers the one with the least time per visibility. Keys are (device, form,
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

// Visibilities a variant is timed on: two full waves of its resident CTAs
// (as many as fit an SM by shared memory and threads; registers may admit
// fewer, which only adds waves), so that small-CTA shapes are measured at
// the occupancy they reach on a large batch, not on a sample that leaves
// SMs idle; at least 131072, at most the whole batch. Variants are compared
// by time per visibility.
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
    for (int v = 0; v < kNumWaveletVariants; ++v) {
        if (!wavelet_variant_fits(v, jb.mode, jb.which, jb.J)) continue;
        sample.n_vis = sample_size(v, jb);
        if (launch_wavelet(sample, v, s) != WT_OK) continue;   // warm-up
        cudaEventRecord(e0, s);
        bool ok = launch_wavelet(sample, v, s) == WT_OK;
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess || !ok) {
            cudaGetLastError();
            continue;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
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
