// wt_api.cu -- the extern "C" boundary of libwtvis: argument checks, handle
// lifetime, error reporting, and dispatch to the kernels. No computation of
// the method happens here; every step runs in the kernels of the other files.
#include <math.h>

#include <cmath>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "wt_internal.cuh"

namespace wt {

namespace {
thread_local char g_msg[512] = "no error";
std::mutex g_mu;
int* g_status[64] = {nullptr};
uint64_t g_status_ctx[64] = {0};   // context ID each status word belongs to
int g_sms[64] = {0};

// cuMemGetAddressRange from the driver, looked up at run time so that the
// library loads on machines without a driver (every call then fails cleanly).
typedef int (*AddrRangeFn)(unsigned long long*, size_t*, unsigned long long);
AddrRangeFn g_addr_range = nullptr;
bool g_addr_range_tried = false;

AddrRangeFn addr_range_fn()
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr_range_tried) {
        g_addr_range_tried = true;
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_addr_range = reinterpret_cast<AddrRangeFn>(fn);
        else
            cudaGetLastError();
    }
    return g_addr_range;
}

// The driver's current context and its unique ID (cuCtxGetCurrent,
// cuCtxGetId), looked up at run time like cuMemGetAddressRange. Caches of
// device memory that belongs to a context are keyed on this ID: a context
// that is destroyed and created again (cudaDeviceReset, or a host framework
// tearing its context down) gets a new ID, and the caches are rebuilt.
typedef int (*CtxGetCurrentFn)(void**);
typedef int (*CtxGetIdFn)(void*, unsigned long long*);
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;
bool g_ctx_tried = false;

void ctx_fns()
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_ctx_tried) return;
    g_ctx_tried = true;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
        g_ctx_current = reinterpret_cast<CtxGetCurrentFn>(fn);
    fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
        g_ctx_id = reinterpret_cast<CtxGetIdFn>(fn);
    cudaGetLastError();
}

int current_device(int* dev)
{
    cudaError_t e = cudaGetDevice(dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    if (*dev < 0 || *dev >= 64) return set_error(WT_ERR_CUDA, "device ordinal %d out of range", *dev);
    return WT_OK;
}
}  // namespace

int set_error(int status, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
    va_end(ap);
    return status;
}

int cuda_error(cudaError_t e, const char* what)
{
    cudaGetLastError();
    return set_error(WT_ERR_CUDA, "%s: %s (%d)", what, cudaGetErrorString(e), static_cast<int>(e));
}

// Unique ID of the current context (made current first if the runtime has
// not done so yet); 0 if there is none.
uint64_t current_context_id()
{
    ctx_fns();
    if (!g_ctx_current || !g_ctx_id) return 0;
    void* ctx = nullptr;
    if (g_ctx_current(&ctx) != 0 || !ctx) {
        cudaFree(nullptr);   // the runtime creates (or makes current) the primary context
        cudaGetLastError();
        ctx = nullptr;
        if (g_ctx_current(&ctx) != 0 || !ctx) return 0;
    }
    unsigned long long id = 0;
    if (g_ctx_id(ctx, &id) != 0) return 0;
    return static_cast<uint64_t>(id) + 1;   // never 0
}

int* device_status_word()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    const uint64_t ctx = current_context_id();
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_status[dev] && g_status_ctx[dev] != ctx) g_status[dev] = nullptr;   // its context is gone
    if (!g_status[dev]) {
        int* p = nullptr;
        if (cudaMalloc(&p, sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        if (cudaMemset(p, 0, sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(p);
            return nullptr;
        }
        g_status[dev] = p;
        g_status_ctx[dev] = ctx;
        // Keep stream-ordered allocations cached in the pool between calls.
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
        cudaGetLastError();
    }
    return g_status[dev];
}

int num_sms()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    if (g_sms[dev] == 0) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        g_sms[dev] = n > 0 ? n : 1;
    }
    return g_sms[dev];
}

// A pointer the kernels will dereference must be device (or managed) memory
// of the current device, and [p, p + bytes) must lie inside its allocation.
int check_device_buffer(const void* p, size_t bytes, const char* fn, const char* name, size_t align)
{
    if (bytes == 0) return WT_OK;
    if (!p) return set_error(WT_ERR_ARG, "%s: %s is NULL", fn, name);
    if (align > 1 && reinterpret_cast<uintptr_t>(p) % align != 0)
        return set_error(WT_ERR_ARG, "%s: %s must be %zu-byte aligned", fn, name, align);
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(WT_ERR_ARG, "%s: %s is not a CUDA pointer (%s)", fn, name, cudaGetErrorString(e));
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return set_error(WT_ERR_ARG, "%s: %s must be device memory", fn, name);
    int dev = 0;
    int rc = current_device(&dev);
    if (rc) return rc;
    if (a.type == cudaMemoryTypeDevice && a.device != dev)
        return set_error(WT_ERR_ARG, "%s: %s lives on device %d, current device is %d", fn, name, a.device, dev);
    AddrRangeFn f = addr_range_fn();
    if (f) {
        unsigned long long base = 0;
        size_t size = 0;
        if (f(&base, &size, reinterpret_cast<unsigned long long>(p)) == 0) {
            const unsigned long long end = base + size;
            const unsigned long long q = reinterpret_cast<unsigned long long>(p);
            if (q + bytes > end)
                return set_error(WT_ERR_ARG, "%s: %s holds %llu bytes from this address, %zu needed", fn, name,
                                 end - q, bytes);
        }
    }
    return WT_OK;
}

}  // namespace wt

using namespace wt;

static int check_tree(wt_tree t, const char* fn)
{
    if (!t) return set_error(WT_ERR_ARG, "%s: tree is NULL", fn);
    if (t->magic != kTreeMagic) return set_error(WT_ERR_CORRUPT, "%s: not a live tree handle", fn);
    int dev = 0;
    int rc = wt::current_device(&dev);
    if (rc) return rc;
    if (dev != t->device)
        return set_error(WT_ERR_ARG, "%s: tree was built on device %d, current device is %d", fn, t->device, dev);
    return WT_OK;
}

namespace {

// A new tree handle built from `src` (checked by the caller).
int new_tree(const char* fn, const wt::KeySource& src, const double* flux, int64_t n_comp, double ra0, double dec0,
             int J, wt_tree* out, void* stream)
{
    int dev = 0;
    int rc;
    if ((rc = wt::current_device(&dev))) return rc;
    wt_tree t = new (std::nothrow) wt_tree_s();
    if (!t) return set_error(WT_ERR_NOMEM, "%s: host allocation failed", fn);
    memset(static_cast<void*>(t), 0, sizeof(*t));
    t->magic = kTreeMagic;
    t->device = dev;
    t->J = J;
    t->ra0 = ra0;
    t->dec0 = dec0;
    t->n_comp = n_comp;
    t->stream = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMallocHost(reinterpret_cast<void**>(&t->host_hdr), sizeof(TreeHeader));
    if (e != cudaSuccess) {
        t->magic = 0;
        delete t;
        return cuda_error(e, "cudaMallocHost");
    }
    rc = wt::build_tree(src, flux, n_comp, ra0, dec0, J, t, t->stream);
    if (rc != WT_OK) {
        if (t->block) cudaFreeAsync(t->block, t->stream);
        cudaStreamSynchronize(t->stream);
        cudaFreeHost(t->host_hdr);
        t->magic = 0;
        delete t;
        return rc;
    }
    *out = t;
    return WT_OK;
}

int check_tree_args(const char* fn, int64_t n_comp, double ra0, double dec0, int J)
{
    if (n_comp < 0) return set_error(WT_ERR_ARG, "%s: n_comp < 0", fn);
    if (n_comp > (int64_t(1) << 30)) return set_error(WT_ERR_RANGE, "%s: n_comp too large", fn);
    if (J < 1 || J > kMaxJ) return set_error(WT_ERR_RANGE, "%s: J = %d outside 1..%d", fn, J, kMaxJ);
    if (!isfinite(ra0) || !isfinite(dec0)) return set_error(WT_ERR_RANGE, "%s: non-finite phase centre", fn);
    return WT_OK;
}

}  // namespace

extern "C" {


int wt_build_tree(const double* l, const double* m, const double* flux, int64_t n_comp, double ra0, double dec0,
                  int J, wt_tree* out, void* stream)
{
    const char* fn = "wt_build_tree";
    if (!out) return set_error(WT_ERR_ARG, "%s: out is NULL", fn);
    *out = nullptr;
    int rc;
    if ((rc = check_tree_args(fn, n_comp, ra0, dec0, J))) return rc;
    const size_t nb = static_cast<size_t>(n_comp) * sizeof(double);
    if ((rc = check_device_buffer(l, nb, fn, "l", 8)) || (rc = check_device_buffer(m, nb, fn, "m", 8)) ||
        (rc = check_device_buffer(flux, nb, fn, "flux", 8)))
        return rc;
    wt::KeySource src;
    src.l = l;
    src.m = m;
    return new_tree(fn, src, flux, n_comp, ra0, dec0, J, out, stream);
}

int wt_tree_import(const int64_t* leaf_keys, const double* leaf_flux, int64_t n_leaves, double ra0, double dec0,
                   int J, wt_tree* out, void* stream)
{
    const char* fn = "wt_tree_import";
    if (!out) return set_error(WT_ERR_ARG, "%s: out is NULL", fn);
    *out = nullptr;
    int rc;
    if ((rc = check_tree_args(fn, n_leaves, ra0, dec0, J))) return rc;
    if (n_leaves > 0 && (!leaf_keys || !leaf_flux)) return set_error(WT_ERR_ARG, "%s: NULL host array", fn);
    // host checks: keys of level J, strictly ascending (distinct), finite fluxes
    const int64_t npix = 12 * (int64_t(1) << (2 * (J - 1)));
    for (int64_t i = 0; i < n_leaves; ++i) {
        if (leaf_keys[i] < 0 || leaf_keys[i] >= npix)
            return set_error(WT_ERR_RANGE, "%s: key %lld is not a level-%d pixel", fn, (long long)leaf_keys[i], J);
        if (i > 0 && leaf_keys[i] <= leaf_keys[i - 1])
            return set_error(WT_ERR_ARG, "%s: keys must be distinct and ascending (at %lld)", fn, (long long)i);
        if (!std::isfinite(leaf_flux[i])) return set_error(WT_ERR_RANGE, "%s: non-finite flux at %lld", fn, (long long)i);
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t kb = static_cast<size_t>(n_leaves > 0 ? n_leaves : 1) * sizeof(int64_t);
    char* d = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&d), 2 * ((kb + 255) & ~size_t(255)), s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(WT_ERR_NOMEM, "%s: scratch allocation failed", fn);
    }
    int64_t* dk = reinterpret_cast<int64_t*>(d);
    double* df = reinterpret_cast<double*>(d + ((kb + 255) & ~size_t(255)));
    if (n_leaves > 0) {
        // pageable host memory: the copies are staged before they return
        e = cudaMemcpyAsync(dk, leaf_keys, static_cast<size_t>(n_leaves) * sizeof(int64_t), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(df, leaf_flux, static_cast<size_t>(n_leaves) * sizeof(double), cudaMemcpyHostToDevice,
                                s);
        if (e != cudaSuccess) {
            cudaFreeAsync(d, s);
            return cuda_error(e, "wt_tree_import: upload");
        }
    }
    wt::KeySource src;
    src.leaf_keys = dk;
    rc = new_tree(fn, src, df, n_leaves, ra0, dec0, J, out, stream);
    cudaFreeAsync(d, s);
    cudaGetLastError();
    return rc;
}

int wt_xref_table(int n, double dl, double ra0, double dec0, int J, int64_t* table, void* stream)
{
    const char* fn = "wt_xref_table";
    if (n < 1 || n > 16384) return set_error(WT_ERR_ARG, "%s: n = %d outside 1..16384", fn, n);
    if (!(dl > 0.0) || !isfinite(dl)) return set_error(WT_ERR_RANGE, "%s: pixel size must be positive", fn);
    if (J < 1 || J > kMaxJ) return set_error(WT_ERR_RANGE, "%s: J = %d outside 1..%d", fn, J, kMaxJ);
    if (!isfinite(ra0) || !isfinite(dec0)) return set_error(WT_ERR_RANGE, "%s: non-finite phase centre", fn);
    int rc;
    if ((rc = check_device_buffer(table, static_cast<size_t>(n) * n * sizeof(int64_t), fn, "table", 8))) return rc;
    return wt::xref_table(n, dl, ra0, dec0, J, table, static_cast<cudaStream_t>(stream));
}

int wt_build_tree_xref(const int64_t* table, int n, const int32_t* pix, const double* flux, int64_t n_comp,
                       double ra0, double dec0, int J, wt_tree* out, void* stream)
{
    const char* fn = "wt_build_tree_xref";
    if (!out) return set_error(WT_ERR_ARG, "%s: out is NULL", fn);
    *out = nullptr;
    int rc;
    if ((rc = check_tree_args(fn, n_comp, ra0, dec0, J))) return rc;
    if (n < 1 || n > 16384) return set_error(WT_ERR_ARG, "%s: n = %d outside 1..16384", fn, n);
    const int64_t nn = static_cast<int64_t>(n) * n;
    if ((rc = check_device_buffer(table, static_cast<size_t>(nn) * sizeof(int64_t), fn, "table", 8)) ||
        (rc = check_device_buffer(pix, static_cast<size_t>(n_comp) * sizeof(int32_t), fn, "pix", 4)) ||
        (rc = check_device_buffer(flux, static_cast<size_t>(n_comp) * sizeof(double), fn, "flux", 8)))
        return rc;
    wt::KeySource src;
    src.table = table;
    src.n_pix = nn;
    src.pix = pix;
    return new_tree(fn, src, flux, n_comp, ra0, dec0, J, out, stream);
}

int wt_tree_info(wt_tree t, int* J, int64_t* n_leaves, int64_t* n_nodes, int64_t* nodes_per_level)
{
    int rc = check_tree(t, "wt_tree_info");
    if (rc) return rc;
    if ((rc = wt::tree_sync_header(t))) return rc;
    const TreeHeader* h = t->host_hdr;
    if (J) *J = t->J;
    if (n_leaves) *n_leaves = h->n_leaves;
    if (n_nodes) *n_nodes = h->n_nodes;
    if (nodes_per_level)
        for (int j = 1; j <= t->J; ++j) nodes_per_level[j - 1] = h->per_level[j];
    return WT_OK;
}

int wt_tree_export(wt_tree t, int64_t* key, uint8_t* child_mask, int32_t* first_child, double* lambda, double* gamma,
                   double* leaf_dir, double* leaf_flux)
{
    int rc = check_tree(t, "wt_tree_export");
    if (rc) return rc;
    if ((rc = wt::tree_sync_header(t))) return rc;
    const TreeHeader h = *t->host_hdr;
    const int64_t T = h.n_nodes, NL = h.n_leaves;
    if (T == 0) return WT_OK;
    const TreeDev& d = t->d;
    std::vector<int64_t> k(T);
    std::vector<uint8_t> mk(T);
    std::vector<int32_t> fc(T);
    std::vector<double> lam(T), gam(3 * T);
    WT_CUDA_TRY(cudaMemcpy(k.data(), d.key, T * sizeof(int64_t), cudaMemcpyDeviceToHost));
    WT_CUDA_TRY(cudaMemcpy(mk.data(), d.mask, T, cudaMemcpyDeviceToHost));
    WT_CUDA_TRY(cudaMemcpy(fc.data(), d.first_child, T * sizeof(int32_t), cudaMemcpyDeviceToHost));
    WT_CUDA_TRY(cudaMemcpy(lam.data(), d.lambda, T * sizeof(double), cudaMemcpyDeviceToHost));
    WT_CUDA_TRY(cudaMemcpy(gam.data(), d.gamma, 3 * T * sizeof(double), cudaMemcpyDeviceToHost));
    // level-J-first layout -> breadth-first (level ascending)
    int64_t bfs_off[kMaxJ + 2];
    bfs_off[1] = 0;
    for (int j = 1; j <= t->J; ++j) bfs_off[j + 1] = bfs_off[j] + h.per_level[j];
    for (int j = 1; j <= t->J; ++j) {
        for (int64_t i = 0; i < h.per_level[j]; ++i) {
            const int64_t src = h.rev_offset[j] + i, dst = bfs_off[j] + i;
            if (key) key[dst] = k[src];
            if (child_mask) child_mask[dst] = mk[src];
            if (first_child) first_child[dst] = (j < t->J) ? static_cast<int32_t>(bfs_off[j + 1] + fc[src]) : -1;
            if (lambda) lambda[dst] = lam[src];
            if (gamma)
                for (int q = 0; q < 3; ++q) gamma[3 * dst + q] = gam[3 * src + q];
        }
    }
    if (leaf_dir) WT_CUDA_TRY(cudaMemcpy(leaf_dir, d.leaf_dir, 3 * NL * sizeof(double), cudaMemcpyDeviceToHost));
    if (leaf_flux) WT_CUDA_TRY(cudaMemcpy(leaf_flux, d.leaf_flux, NL * sizeof(double), cudaMemcpyDeviceToHost));
    return WT_OK;
}

void wt_free_tree(wt_tree t)
{
    if (!t || t->magic != kTreeMagic) return;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != t->device) cudaSetDevice(t->device);
    wt::batch_forget_tree(t);
    cudaStreamSynchronize(t->stream);
    if (t->block) cudaFreeAsync(t->block, t->stream);
    cudaStreamSynchronize(t->stream);
    if (t->host_hdr) cudaFreeHost(t->host_hdr);
    cudaGetLastError();
    if (prev >= 0 && prev != t->device) cudaSetDevice(prev);
    t->magic = 0;
    delete t;
}

int wt_predict_vis(wt_tree t, const double* uvw, int64_t n_vis, void* vis_out, int mode, int sign, int which,
                   void* stream)
{
    const char* fn = "wt_predict_vis";
    int rc = check_tree(t, fn);
    if (rc) return rc;
    if (n_vis < 0) return set_error(WT_ERR_ARG, "%s: n_vis < 0", fn);
    if (sign != 1 && sign != -1) return set_error(WT_ERR_ARG, "%s: sign must be +1 or -1", fn);
    if (which != WT_SUM_EQ17 && which != WT_SUM_EQ16 && which != WT_SUM_EQ17_REGROUPED)
        return set_error(WT_ERR_ARG, "%s: bad sum selector", fn);
    if (mode == WT_LEARNED)
        return set_error(WT_ERR_UNSUPPORTED, "%s: the learned response has its own entry point", fn);
    if (mode != WT_FP64 && mode != WT_MIXED && mode != WT_MIXED_FAST && mode != WT_FP64_DF && mode != WT_MIXED_TC)
        return set_error(WT_ERR_ARG, "%s: bad mode %d", fn, mode);
    if (mode == WT_FP64_DF && which == WT_SUM_EQ17)
        return set_error(WT_ERR_UNSUPPORTED, "%s: WT_FP64_DF evaluates the regrouped Eq. 17 and Eq. 16 only", fn);
    const size_t ob = static_cast<size_t>(n_vis) * ((mode == WT_FP64 || mode == WT_FP64_DF) ? 16 : 8);
    if ((rc = check_device_buffer(uvw, static_cast<size_t>(n_vis) * 24, fn, "uvw", 8)) ||
        (rc = check_device_buffer(vis_out, ob, fn, "vis_out", vis_align(mode))))
        return rc;
    return wt::predict_wavelet(t, uvw, n_vis, vis_out, mode, sign, which, static_cast<cudaStream_t>(stream));
}

int dft_predict_vis(const double* l, const double* m, const double* flux, int64_t n_comp, const double* uvw,
                    int64_t n_vis, void* vis_out, int mode, int sign, void* stream)
{
    const char* fn = "dft_predict_vis";
    if (n_comp < 0 || n_vis < 0) return set_error(WT_ERR_ARG, "%s: negative size", fn);
    if (n_comp > (int64_t(1) << 30)) return set_error(WT_ERR_RANGE, "%s: n_comp too large", fn);
    if (sign != 1 && sign != -1) return set_error(WT_ERR_ARG, "%s: sign must be +1 or -1", fn);
    if (mode != WT_FP64 && mode != WT_MIXED && mode != WT_MIXED_FAST && mode != WT_FP64_DF && mode != WT_MIXED_TC)
        return set_error(WT_ERR_ARG, "%s: bad mode %d", fn, mode);
    const size_t nb = static_cast<size_t>(n_comp) * 8;
    const size_t ob = static_cast<size_t>(n_vis) * ((mode == WT_FP64 || mode == WT_FP64_DF) ? 16 : 8);
    int rc;
    if ((rc = check_device_buffer(l, nb, fn, "l", 8)) || (rc = check_device_buffer(m, nb, fn, "m", 8)) ||
        (rc = check_device_buffer(flux, nb, fn, "flux", 8)) ||
        (rc = check_device_buffer(uvw, static_cast<size_t>(n_vis) * 24, fn, "uvw", 8)) ||
        (rc = check_device_buffer(vis_out, ob, fn, "vis_out", vis_align(mode))))
        return rc;
    if (!device_status_word()) return set_error(WT_ERR_CUDA, "%s: no usable CUDA device", fn);
    return wt::predict_dft(l, m, flux, n_comp, uvw, n_vis, vis_out, mode, sign, static_cast<cudaStream_t>(stream));
}

int subtract_model(const void* vis_obs, const void* vis_model, void* vis_resid, int64_t n_vis, int mode, void* stream)
{
    const char* fn = "subtract_model";
    if (n_vis < 0) return set_error(WT_ERR_ARG, "%s: n_vis < 0", fn);
    if (mode != WT_FP64 && mode != WT_MIXED && mode != WT_LEARNED && mode != WT_MIXED_FAST && mode != WT_FP64_DF &&
        mode != WT_MIXED_TC)
        return set_error(WT_ERR_ARG, "%s: bad mode", fn);
    if (mode == WT_FP64_DF) mode = WT_FP64;   // both complex128
    const size_t b = static_cast<size_t>(n_vis) * (mode == WT_FP64 ? 16 : 8);
    int rc;
    const size_t al = vis_align(mode);   // complex64 views need not be 16-byte aligned (a scalar path takes them)
    if ((rc = check_device_buffer(vis_obs, b, fn, "vis_obs", al)) ||
        (rc = check_device_buffer(vis_model, b, fn, "vis_model", al)) ||
        (rc = check_device_buffer(vis_resid, b, fn, "vis_resid", al)))
        return rc;
    if (!device_status_word()) return set_error(WT_ERR_CUDA, "%s: no usable CUDA device", fn);
    return wt::subtract(vis_obs, vis_model, vis_resid, n_vis, mode, static_cast<cudaStream_t>(stream));
}

int wt_recommended_J(double dtheta_rad)
{
    if (!(dtheta_rad > 0.0) || !isfinite(dtheta_rad)) return set_error(WT_ERR_ARG, "wt_recommended_J: dtheta <= 0");
    for (int J = 1; J <= kMaxJ; ++J) {
        const double pix = ldexp(sqrt(kPi / 3.0), 1 - J);   // Delta theta_J
        if (pix <= 0.5 * dtheta_rad) return J;
    }
    return set_error(WT_ERR_RANGE, "wt_recommended_J: needs J > %d", kMaxJ);
}

int wt_device_status(void* stream)
{
    int* w = device_status_word();
    if (!w) return set_error(WT_ERR_CUDA, "wt_device_status: no usable CUDA device");
    WT_CUDA_TRY(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    int v = 0;
    WT_CUDA_TRY(cudaMemcpy(&v, w, sizeof(int), cudaMemcpyDeviceToHost));
    if (v != 0) {
        WT_CUDA_TRY(cudaMemset(w, 0, sizeof(int)));
        return set_error(v, "a kernel reported status %d", v);
    }
    return WT_OK;
}

const char* wt_last_error(void) { return g_msg; }

}  // extern "C"

namespace wt {
// One CTA waits on an mbarrier whose phase never completes (nothing arrives
// on it), with `limit` polls: the wait must give up and report
// WT_ERR_TIMEOUT through the status word, and the kernel return normally.
__global__ void k_selftest_bounded_wait(uint32_t limit, int* status)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        wt::mbar_init(&bar, 1);
        wt::fence_mbar_init();
    }
    __syncthreads();
    const bool ok = wt::mbar_wait_parity(&bar, 0, limit);
    if (!__syncthreads_and(ok ? 1 : 0) && threadIdx.x == 0) wt::record_status(status, WT_ERR_TIMEOUT);
}
}  // namespace wt

extern "C" {

int wt_selftest_bounded_wait(uint32_t spin_limit, void* stream)
{
    if (spin_limit == 0 || spin_limit > (1u << 16))
        return set_error(WT_ERR_ARG, "wt_selftest_bounded_wait: spin_limit must be in 1..65536");
    int* w = device_status_word();
    if (!w) return set_error(WT_ERR_CUDA, "wt_selftest_bounded_wait: no usable CUDA device");
    wt::k_selftest_bounded_wait<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(spin_limit, w);
    WT_CUDA_TRY(cudaGetLastError());
    return WT_OK;
}

}  // extern "C"
