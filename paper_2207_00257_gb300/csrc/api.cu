// api.cu -- the C ABI of include/gbconv.h: argument validation, dispatch to
// the CUDA-core and tensor-core kernels, the device error word, and the
// tuning table (in memory, JSON on disk).
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"

// The one device word every bounded in-kernel wait reports to (static device
// memory: nothing is allocated for it).
__device__ unsigned int g_gbconv_error_word;

// Scratch of conv2d_dgrad_noalloc: the rotated filter lives here instead of in
// a caller's workspace. Every GPU that loads the library holds it until exit.
static __device__ __align__(256) unsigned char g_dgrad_static_scratch[GBCONV_DGRAD_STATIC_SCRATCH_BYTES];

namespace gbc {
// Reads a tuning-table JSON file into the table (defined below the C ABI).
gbconv_status_t load_cache_file(const char *path);

namespace {

std::mutex g_mu;
int g_skip_loads = 0;

// Environment settings, read once:
//   GBCONV_WAIT_LIMIT  default time limit of every in-kernel wait, in ns
//                      (default 2e9);
//   GBCONV_TUNE_CACHE  path of a tuning-table JSON file: loaded on the first
//                      lookup, rewritten after every gbconv_tune;
//   GBCONV_LOG         0 (default) silent, 1 failed calls, 2 every call's
//                      problem and configuration, on stderr.
uint64_t env_u64(const char *name, uint64_t dflt) {
    const char *v = getenv(name);
    if (!v || !*v) return dflt;
    char *end = nullptr;
    unsigned long long x = strtoull(v, &end, 10);
    return (end && *end == 0 && x > 0) ? (uint64_t)x : dflt;
}
uint64_t default_wait_ns() {
    static const uint64_t v = env_u64("GBCONV_WAIT_LIMIT", 2000000000ull);
    return v;
}
int log_level() {
    static const int v = (int)env_u64("GBCONV_LOG", 0);
    return v;
}
uint64_t g_wait_ns = default_wait_ns();

void log_call(const char *what, const gbconv_problem_t *p, const TcConfig *c, gbconv_status_t st) {
    const int lv = log_level();
    if (lv <= 0 || (lv == 1 && st == GBCONV_OK) || !p) return;
    fprintf(stderr,
            "[gbconv] %s N=%d C=%d H=%d W=%d K=%d R=%d S=%d stride=%d,%d pad=%d,%d dil=%d,%d "
            "in=%d out=%d layout=%d flags=%u groups=%d",
            what, p->N, p->C, p->H, p->W, p->K, p->R, p->S, p->stride_h, p->stride_w, p->pad_h,
            p->pad_w, p->dil_h, p->dil_w, p->in_dtype, p->out_dtype, p->layout, p->flags, p->groups);
    if (c)
        fprintf(stderr, " block_n=%d stages=%d split_k=%d raster=%d algo=%d", c->block_n, c->stages,
                c->split_k, c->raster, c->algo);
    fprintf(stderr, " -> %d\n", (int)st);
}

struct DevInfo {
    unsigned int *err = nullptr;
    int sms = 0;
    std::string name;
    bool init = false;
};
constexpr int MAX_DEV = 64;
DevInfo g_dev[MAX_DEV];

DevInfo *dev_info() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEV) return nullptr;
    std::lock_guard<std::mutex> lock(g_mu);
    DevInfo &di = g_dev[dev];
    if (!di.init) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_gbconv_error_word) != cudaSuccess) return nullptr;
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return nullptr;
        cudaDeviceProp prop;
        if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return nullptr;
        di.err = static_cast<unsigned int *>(p);
        di.sms = sms;
        di.name = prop.name;
        di.init = true;
    }
    return &di;
}

// ---- tuning table ----
std::map<std::string, TcConfig> g_tune;

std::string problem_key(int op, const gbconv_problem_t &p) {
    DevInfo *di = dev_info();
    char buf[512];
    snprintf(buf, sizeof buf, "%d|%d,%d,%d,%d,%d,%d,%d|%d,%d,%d,%d,%d,%d|%d,%d,%d,%u|g%d|%s", op,
             p.N, p.C, p.H, p.W, p.K, p.R, p.S, p.stride_h, p.stride_w, p.pad_h, p.pad_w, p.dil_h,
             p.dil_w, p.in_dtype, p.out_dtype, p.layout, p.flags, p.groups > 1 ? p.groups : 1,
             di ? di->name.c_str() : "?");
    return buf;
}

void load_env_cache_once() {
    static std::once_flag once;
    std::call_once(once, []() {
        const char *path = getenv("GBCONV_TUNE_CACHE");
        if (path && *path) {
            FILE *f = fopen(path, "r");
            if (f) {
                fclose(f);
                if (load_cache_file(path) != GBCONV_OK && log_level() > 0)
                    fprintf(stderr, "[gbconv] could not parse GBCONV_TUNE_CACHE=%s\n", path);
            }
        }
    });
}

bool tuned(int op, const gbconv_problem_t &p, TcConfig *out) {
    load_env_cache_once();
    std::string k = problem_key(op, p);
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_tune.find(k);
    if (it == g_tune.end()) return false;
    *out = it->second;
    return true;
}

// ---- validation ----
gbconv_status_t make_dims(const gbconv_problem_t *p, Dims *d) {
    if (!p) return GBCONV_ERR_INVALID_ARG;
    if (p->N < 0 || p->C < 1 || p->H < 1 || p->W < 1 || p->K < 1 || p->R < 1 || p->S < 1)
        return GBCONV_ERR_INVALID_ARG;
    if (p->stride_h < 1 || p->stride_w < 1 || p->dil_h < 1 || p->dil_w < 1 || p->pad_h < 0 ||
        p->pad_w < 0)
        return GBCONV_ERR_INVALID_ARG;
    if (p->in_dtype < GBCONV_F32 || p->in_dtype > GBCONV_E4M3 || p->out_dtype < GBCONV_F32 ||
        p->out_dtype > GBCONV_E4M3 || (p->layout != GBCONV_NCHW && p->layout != GBCONV_NHWC))
        return GBCONV_ERR_INVALID_ARG;
    if (p->flags & ~(GBCONV_FLAG_BIAS | GBCONV_FLAG_RELU)) return GBCONV_ERR_INVALID_ARG;
    const int G = p->groups > 1 ? p->groups : 1;
    if (p->groups < 0 || p->C % G != 0 || p->K % G != 0) return GBCONV_ERR_INVALID_ARG;
    long long pn = (long long)p->H + 2ll * p->pad_h - (long long)p->dil_h * (p->R - 1) - 1;
    long long qn = (long long)p->W + 2ll * p->pad_w - (long long)p->dil_w * (p->S - 1) - 1;
    if (pn < 0 || qn < 0) return GBCONV_ERR_INVALID_ARG;
    d->N = p->N;
    d->C = p->C;
    d->H = p->H;
    d->W = p->W;
    d->K = p->K;
    d->R = p->R;
    d->S = p->S;
    d->P = (int)(pn / p->stride_h + 1);
    d->Q = (int)(qn / p->stride_w + 1);
    d->u = p->stride_h;
    d->v = p->stride_w;
    d->ph = p->pad_h;
    d->pw = p->pad_w;
    d->dh = p->dil_h;
    d->dw = p->dil_w;
    d->layout = p->layout;
    d->in_dtype = p->in_dtype;
    d->out_dtype = p->out_dtype;
    d->flags = p->flags;
    d->G = G;
    // element counts must fit the kernels' 64-bit offsets comfortably
    const long long lim = 1ll << 40;
    if ((long long)d->N * d->C * d->H * d->W >= lim || (long long)d->N * d->K * d->P * d->Q >= lim ||
        (long long)d->K * d->C * d->R * d->S >= lim)
        return GBCONV_ERR_INVALID_ARG;
    return GBCONV_OK;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }


// Tensor-core forward eligibility beyond tc_fwd_supported: argument-level checks.
gbconv_status_t check_tc_fwd(const Dims &d, const void *x, const void *w, const void *y) {
    if (d.in_dtype == GBCONV_BF16 && (d.C % 8 || d.K % 8)) return GBCONV_ERR_ALIGNMENT;
    if (d.in_dtype == GBCONV_E4M3 && (d.C % 16 || d.K % 8)) return GBCONV_ERR_ALIGNMENT;
    if (!aligned16(x) || !aligned16(w) || !aligned16(y)) return GBCONV_ERR_ALIGNMENT;
    if (!tc_fwd_supported(d)) return GBCONV_ERR_UNSUPPORTED;
    return GBCONV_OK;
}

// The data gradient of a stride-1 convolution is a forward convolution of dy
// with the filter rotated by 180 degrees (C and K exchanged) and padding
// dil*(R-1) - pad: dx[n,h,w,c] = sum_{k,r',s'} dy[n, h - (pad' ) + r' d, ...] w_rot.
bool dgrad_as_fwd(const Dims &d, Dims *t) {
    if (d.layout != GBCONV_NHWC || d.in_dtype != GBCONV_BF16) return false;
    if (d.u != 1 || d.v != 1) return false;
    const int ph2 = d.dh * (d.R - 1) - d.ph, pw2 = d.dw * (d.S - 1) - d.pw;
    if (ph2 < 0 || pw2 < 0) return false;
    Dims e = d;
    e.C = d.K;
    e.K = d.C;
    e.H = d.P;
    e.W = d.Q;
    e.ph = ph2;
    e.pw = pw2;
    e.P = d.H;
    e.Q = d.W;
    e.flags = 0;
    e.in_dtype = GBCONV_BF16;
    e.out_dtype = d.out_dtype;
    if (e.C % 8 || e.K % 8 || !tc_fwd_supported(e)) return false;
    *t = e;
    return true;
}

size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

int wgrad_default_slices(const Dims &d) {
    // about eight CTAs per SM of a 152-SM part, at most 64 slices, and no
    // more slices than the reduction has 16-pixel runs
    long long tiles = (long long)d.G * ((d.K / d.G + 127) / 128) * ((d.C / d.G + 63) / 64) * d.R * d.S;
    long long runs = (long long)d.N * d.P * ((d.Q + 15) / 16);
    long long s = (1216 + tiles - 1) / tiles;
    s = std::min<long long>(s, 64);
    s = std::min<long long>(s, std::max<long long>(runs, 1));
    return (int)std::max<long long>(s, 1);
}

TcConfig config_for(int op, const gbconv_problem_t &p, const Dims &d) {
    TcConfig c{};
    if (tuned(op, p, &c)) return c;
    if (op == GBCONV_OP_GROUPED) return tc_fwd_default_config(d);  // untuned: the forward heuristic
    if (op == GBCONV_OP_WGRAD) {
        if (d.G == 1 && tc_wgrad_supported(d)) return tc_wgrad_default_config(d);
        c.split_k = wgrad_default_slices(d);
        return c;
    }
    if (op == GBCONV_OP_DGRAD) {
        Dims t;
        if (d.G == 1 && dgrad_as_fwd(d, &t)) return tc_fwd_default_config(t);
        return c;
    }
    if (tc_fwd_supported(d)) return tc_fwd_default_config(d);
    return c;
}

// Bias-gradient partial sums: a fixed number of row slices, independent of
// the weight gradient's split.
constexpr int BIAS_SLICES = 304;  // 2 x 152 SMs

size_t wgrad_ws_bytes(const Dims &d, int slices) {
    size_t kcrs = (size_t)d.K * (d.C / d.G) * d.R * d.S;
    return round256(((size_t)slices * kcrs + (size_t)BIAS_SLICES * d.K) * sizeof(float));
}

// Forward of a layer with channel groups (d.G > 1): depthwise kernel, one
// persistent tensor-core launch over the groups as separate problems (BF16
// NHWC, C/G and K/G multiples of 8, no fused scale or residual), else the
// CUDA-core implicit GEMM per group.
gbconv_status_t do_fwd_groups(const Dims &d, const void *x, const void *w, const float *bias,
                              const float *x_scale, const float *w_scale, void *y,
                              cudaStream_t st, const Fused &fz) {
    (void)x_scale;
    (void)w_scale;
    if (d.in_dtype == GBCONV_E4M3) return GBCONV_ERR_UNSUPPORTED;
    if (d.in_dtype == GBCONV_F32 && d.out_dtype != GBCONV_F32) return GBCONV_ERR_UNSUPPORTED;
    const int Cg = d.C / d.G, Kg = d.K / d.G;
    if (depthwise_supported(d) && aligned16(x) && aligned16(y) && (!fz.z || aligned16(fz.z)))
        return launch_depthwise(d, x, w, bias, y, st, fz);
    if (d.in_dtype == GBCONV_BF16 && d.layout == GBCONV_NHWC && Cg % 8 == 0 && Kg % 8 == 0 &&
        !fz.alpha && !fz.z && aligned16(x) && aligned16(w) && aligned16(y)) {
        const int ebo = d.out_dtype == GBCONV_F32 ? 4 : 2;
        std::vector<Dims> dg(d.G, d);
        std::vector<TcConfig> cfg(d.G);
        std::vector<const void *> xs(d.G), ws(d.G);
        std::vector<const float *> bs(d.G);
        std::vector<void *> ys(d.G);
        for (int g = 0; g < d.G; ++g) {
            Dims &e = dg[g];
            e.C = Cg;
            e.K = Kg;
            e.G = 1;
            e.ldxc = d.C;
            e.ldyc = d.K;
            cfg[g] = tc_fwd_default_config(e);
            xs[g] = static_cast<const char *>(x) + (size_t)g * Cg * 2;
            ws[g] = static_cast<const char *>(w) + (size_t)g * Kg * d.R * d.S * Cg * 2;
            bs[g] = ((d.flags & GBCONV_FLAG_BIAS) && bias) ? bias + (size_t)g * Kg : nullptr;
            ys[g] = static_cast<char *>(y) + (size_t)g * Kg * ebo;
        }
        return launch_tc_grouped(d.G, dg.data(), cfg.data(), xs.data(), ws.data(), bs.data(),
                                 ys.data(), st);
    }
    return launch_simt_fwd(d, x, w, bias, y, st, fz);
}

// Workspace of a BF16 NCHW forward: x as NHWC, w as KRSC, y as NHWC.
bool nchw_bf16(const Dims &d) {
    return d.layout == GBCONV_NCHW && d.in_dtype == GBCONV_BF16 && d.G == 1;
}
size_t nchw_ws_bytes(const Dims &d) {
    const int eo = d.out_dtype == GBCONV_F32 ? 4 : 2;
    return round256((size_t)d.N * d.H * d.W * d.C * 2) + round256((size_t)d.K * d.R * d.S * d.C * 2) +
           round256((size_t)d.M() * d.K * eo);
}

gbconv_status_t do_fwd(const Dims &d, const TcConfig &cfg, const void *x, const void *w,
                       const float *bias, const float *x_scale, const float *w_scale, void *y,
                       cudaStream_t st, const Fused &fz = Fused{});

// BF16 NCHW forward on the NHWC tensor-core path through layout transforms
// (a transpose kernel in front of the producer and behind the epilogue). The
// residual, if any, is transposed into the NHWC output buffer and added in
// place.
gbconv_status_t do_fwd_nchw_bf16(const Dims &d, const void *x, const void *w, const float *bias,
                                 void *y, void *ws, size_t ws_bytes, cudaStream_t st,
                                 const Fused &fz) {
    if (d.M() == 0) return GBCONV_OK;
    if (!ws || ws_bytes < nchw_ws_bytes(d)) return GBCONV_ERR_WORKSPACE;
    if (!aligned16(ws)) return GBCONV_ERR_ALIGNMENT;
    const int eo = d.out_dtype == GBCONV_F32 ? 4 : 2;
    char *p = static_cast<char *>(ws);
    void *xn = p;
    p += round256((size_t)d.N * d.H * d.W * d.C * 2);
    void *wn = p;
    p += round256((size_t)d.K * d.R * d.S * d.C * 2);
    void *yn = p;
    gbconv_status_t s = launch_transpose_b(x, xn, d.N, d.C, d.H * d.W, 2, st);  // NCHW -> NHWC
    if (s != GBCONV_OK) return s;
    s = launch_transpose_b(w, wn, d.K, d.C, d.R * d.S, 2, st);  // KCRS -> KRSC
    if (s != GBCONV_OK) return s;
    Fused f2 = fz;
    if (fz.z) {  // residual [N][K][P*Q] -> [N][P*Q][K] in the output buffer
        s = launch_transpose_b(fz.z, yn, d.N, d.K, d.P * d.Q, eo, st);
        if (s != GBCONV_OK) return s;
        f2.z = yn;
    }
    Dims e = d;
    e.layout = GBCONV_NHWC;
    s = do_fwd(e, tc_fwd_default_config(e), xn, wn, bias, nullptr, nullptr, yn, st, f2);
    if (s != GBCONV_OK) return s;
    return launch_transpose_b(yn, y, d.N, d.P * d.Q, d.K, eo, st);  // NHWC -> NCHW
}

gbconv_status_t do_fwd(const Dims &d, const TcConfig &cfg, const void *x, const void *w,
                       const float *bias, const float *x_scale, const float *w_scale, void *y,
                       cudaStream_t st, const Fused &fz) {
    if (d.M() == 0) return GBCONV_OK;
    if (d.G > 1) return do_fwd_groups(d, x, w, bias, x_scale, w_scale, y, st, fz);
    if (d.in_dtype == GBCONV_F32) {
        if (d.out_dtype != GBCONV_F32) return GBCONV_ERR_UNSUPPORTED;
        if (cfg.algo != GBCONV_ALGO_SIMT && simt_fast_supported(d, x, w, y, fz.z))
            return launch_simt_fast_fwd(d, x, w, bias, y, st, fz);
        return launch_simt_fwd(d, x, w, bias, y, st, fz);
    }
    if (cfg.algo == GBCONV_ALGO_SIMT) {  // the CUDA-core kernel on request (BF16 in)
        if (d.in_dtype != GBCONV_BF16) return GBCONV_ERR_UNSUPPORTED;
        return launch_simt_fwd(d, x, w, bias, y, st, fz);
    }
    if (d.layout != GBCONV_NHWC) return GBCONV_ERR_UNSUPPORTED;
    if (d.in_dtype == GBCONV_E4M3 && (!x_scale || !w_scale)) return GBCONV_ERR_INVALID_ARG;
    gbconv_status_t s = check_tc_fwd(d, x, w, y);
    if (s != GBCONV_OK) return s;
    if (fz.z && !aligned16(fz.z)) return GBCONV_ERR_ALIGNMENT;  // 16-byte residual loads
    return launch_tc_fwd(d, cfg, x, w, bias, x_scale, w_scale, y, st, fz);
}

gbconv_status_t do_dgrad(const Dims &d, const TcConfig &cfg, const void *dy, const void *w,
                         void *dx, void *ws, size_t ws_bytes, cudaStream_t st) {
    if ((long long)d.N * d.H * d.W == 0) return GBCONV_OK;
    if (d.in_dtype == GBCONV_E4M3 || d.out_dtype == GBCONV_E4M3) return GBCONV_ERR_UNSUPPORTED;
    if (d.in_dtype == GBCONV_F32 && d.out_dtype != GBCONV_F32) return GBCONV_ERR_UNSUPPORTED;
    // channel groups, and the CUDA-core kernel on request
    if (d.G > 1 || cfg.algo == GBCONV_ALGO_SIMT) return launch_simt_dgrad(d, dy, w, dx, st);
    Dims t;
    if (dgrad_as_fwd(d, &t)) {
        size_t need = round256((size_t)d.K * d.R * d.S * d.C * 2);
        if (!ws || ws_bytes < need) return GBCONV_ERR_WORKSPACE;
        if (!aligned16(ws) || !aligned16(dy) || !aligned16(dx)) return GBCONV_ERR_ALIGNMENT;
        gbconv_status_t s = launch_rotate_filter(d, w, ws, st);
        if (s != GBCONV_OK) return s;
        return launch_tc_fwd(t, cfg, dy, ws, nullptr, nullptr, nullptr, dx, st);
    }
    if (tc_dgrad_t_supported(d)) {
        // strided (or over-padded) layer: sub-pixel phases on tensor cores with
        // the transposed filter in the workspace
        size_t need = round256((size_t)d.K * d.R * d.S * d.C * 2);
        if (!ws || ws_bytes < need) return GBCONV_ERR_WORKSPACE;
        if (!aligned16(ws) || !aligned16(dy) || !aligned16(dx)) return GBCONV_ERR_ALIGNMENT;
        gbconv_status_t s = launch_transpose_filter(d, w, ws, st);
        if (s != GBCONV_OK) return s;
        return launch_tc_dgrad_t(d, dy, ws, dx, st);
    }
    return launch_simt_dgrad(d, dy, w, dx, st);
}

gbconv_status_t do_wgrad(const Dims &d, const TcConfig &cfg, const void *x, const void *dy,
                         float *dw, float *db, void *ws, size_t ws_bytes, cudaStream_t st) {
    if (d.in_dtype == GBCONV_E4M3) return GBCONV_ERR_UNSUPPORTED;
    const long long kcrs = (long long)d.K * (d.C / d.G) * d.R * d.S;  // the filter holds C/G channels
    // tensor-core kernels: the per-tap im2col kernel (algo AUTO / IM2COL) or,
    // on request (algo SHIFT), the band kernel; GBCONV_ALGO_SIMT asks for the
    // CUDA-core kernel
    const bool al = aligned16(x) && aligned16(dy) && aligned16(ws);
    const bool band = d.G == 1 && al && cfg.algo == GBCONV_ALGO_SHIFT && tc_wgrad_shift_supported(d);
    const bool tc = !band && d.G == 1 && al && cfg.algo != GBCONV_ALGO_SIMT && tc_wgrad_supported(d);
    int slices = cfg.split_k > 0 ? cfg.split_k : (band ? tc_wgrad_shift_default_slices(d) : 1);
    if (slices > 1024) return GBCONV_ERR_INVALID_ARG;
    // the tensor-core kernels give every slice at least one reduction step
    if (band) slices = (int)std::max<long long>(1, std::min<long long>(slices, tc_wgrad_shift_bands(d)));
    if (tc) slices = (int)std::max<long long>(1, std::min<long long>(slices, tc_wgrad_pixel_steps(d)));
    size_t need = wgrad_ws_bytes(d, slices);
    if (!ws || ws_bytes < need) return GBCONV_ERR_WORKSPACE;
    float *part = static_cast<float *>(ws);
    float *bpart = part + (size_t)slices * kcrs;
    if (d.M() == 0) {
        cudaError_t e = cudaMemsetAsync(dw, 0, kcrs * sizeof(float), st);
        if (e == cudaSuccess && db) e = cudaMemsetAsync(db, 0, d.K * sizeof(float), st);
        return cuda_status(e);
    }
    gbconv_status_t s;
    if (band) {
        s = launch_tc_wgrad_shift_partials(d, slices, x, dy, part, st);
    } else if (tc) {
        TcConfig c = cfg;
        c.split_k = slices;
        s = launch_tc_wgrad_partials(d, c, x, dy, part, st);
    } else
        s = launch_simt_wgrad_partials(d, x, dy, part, slices, st);
    if (s != GBCONV_OK) return s;
    s = launch_reduce_slices(part, slices, kcrs, dw, st);
    if (s != GBCONV_OK) return s;
    if (db) s = launch_bias_grad(d, dy, db, bpart, BIAS_SLICES, st);
    return s;
}

}  // namespace

gbconv_status_t cuda_status(cudaError_t e) { return e == cudaSuccess ? GBCONV_OK : GBCONV_ERR_CUDA; }

Guard make_guard() {
    DevInfo *di = dev_info();
    Guard g;
    g.err = di ? di->err : nullptr;
    g.wait_ns = g_wait_ns;
    g.skip_loads = g_skip_loads;
    return g;
}

int sm_count() {
    DevInfo *di = dev_info();
    return di && di->sms > 0 ? di->sms : 1;
}

}  // namespace gbc

using namespace gbc;

extern "C" {

gbconv_status_t gbconv_output_dims(const gbconv_problem_t *prob, int32_t *P, int32_t *Q) {
    Dims d;
    gbconv_status_t s = make_dims(prob, &d);
    if (s != GBCONV_OK) return s;
    if (!P || !Q) return GBCONV_ERR_INVALID_ARG;
    *P = d.P;
    *Q = d.Q;
    return GBCONV_OK;
}

gbconv_status_t gbconv_workspace_size(int32_t op, const gbconv_problem_t *prob, size_t *bytes) {
    Dims d;
    gbconv_status_t s = make_dims(prob, &d);
    if (s != GBCONV_OK) return s;
    if (!bytes) return GBCONV_ERR_INVALID_ARG;
    *bytes = 0;
    if (op == GBCONV_OP_FWD) {
        if (nchw_bf16(d)) *bytes = nchw_ws_bytes(d);
        return GBCONV_OK;
    }
    if (op == GBCONV_OP_DGRAD) {
        Dims t;
        if (d.G == 1 && (dgrad_as_fwd(d, &t) || tc_dgrad_t_supported(d)))
            *bytes = round256((size_t)d.K * d.R * d.S * d.C * 2);
        return GBCONV_OK;
    }
    if (op == GBCONV_OP_WGRAD) {
        TcConfig c = config_for(op, *prob, d);
        *bytes = wgrad_ws_bytes(d, std::max(1, c.split_k));
        return GBCONV_OK;
    }
    if (op == GBCONV_OP_GROUPED) return GBCONV_OK;  // no workspace
    return GBCONV_ERR_INVALID_ARG;
}

gbconv_status_t conv2d_fwd(const gbconv_problem_t *prob, const void *x, const void *w,
                           const float *bias, const float *x_scale, const float *w_scale, void *y,
                           void *ws, size_t ws_bytes, gbconv_stream_t stream) {
    Dims d;
    gbconv_status_t s = make_dims(prob, &d);
    if (s != GBCONV_OK) return s;
    if (d.N == 0) return GBCONV_OK;  // empty batch: nothing to read or write
    if (!x || !w || !y || ((d.flags & GBCONV_FLAG_BIAS) && !bias)) return GBCONV_ERR_INVALID_ARG;
    if (x == y || w == y) return GBCONV_ERR_INVALID_ARG;
    if (nchw_bf16(d)) {
        s = do_fwd_nchw_bf16(d, x, w, bias, y, ws, ws_bytes, static_cast<cudaStream_t>(stream),
                             Fused{});
        log_call("conv2d_fwd", prob, nullptr, s);
        return s;
    }
    const TcConfig c = config_for(GBCONV_OP_FWD, *prob, d);
    s = do_fwd(d, c, x, w, bias, x_scale, w_scale, y, static_cast<cudaStream_t>(stream));
    log_call("conv2d_fwd", prob, &c, s);
    return s;
}

gbconv_status_t conv2d_fwd_fused(const gbconv_problem_t *prob, const void *x, const void *w,
                                 const float *bias, const float *scale, const void *residual,
                                 const float *x_scale, const float *w_scale, void *y, void *ws,
                                 size_t ws_bytes, gbconv_stream_t stream) {
    Dims d;
    gbconv_status_t s = make_dims(prob, &d);
    if (s != GBCONV_OK) return s;
    if (d.N == 0) return GBCONV_OK;
    if (!x || !w || !y || ((d.flags & GBCONV_FLAG_BIAS) && !bias)) return GBCONV_ERR_INVALID_ARG;
    if (x == y || w == y || residual == x || residual == w) return GBCONV_ERR_INVALID_ARG;
    Fused fz;
    fz.alpha = scale;
    fz.z = residual;
    if (nchw_bf16(d))
        return do_fwd_nchw_bf16(d, x, w, bias, y, ws, ws_bytes, static_cast<cudaStream_t>(stream),
                                fz);
    return do_fwd(d, config_for(GBCONV_OP_FWD, *prob, d), x, w, bias, x_scale, w_scale, y,
                  static_cast<cudaStream_t>(stream), fz);
}

gbconv_status_t gbconv_nll_workspace_size(int64_t N, size_t *bytes) {
    if (N < 0 || !bytes) return GBCONV_ERR_INVALID_ARG;
    *bytes = nll_workspace_bytes(N);
    return GBCONV_OK;
}

gbconv_status_t gbconv_nll_loss_fwd(const float *logp, const int64_t *target, const float *weight,
                                    int64_t N, int64_t C, int64_t ignore_index, int32_t reduction,
                                    float *out, float *total_weight, void *ws, size_t ws_bytes,
                                    gbconv_stream_t stream) {
    if (N < 0 || C < 1 || reduction < 0 || reduction > 2 || !out || !total_weight)
        return GBCONV_ERR_INVALID_ARG;
    if (N > 0 && (!logp || !target)) return GBCONV_ERR_INVALID_ARG;
    if (N * C >= (1ll << 40)) return GBCONV_ERR_INVALID_ARG;
    if (!ws || ws_bytes < nll_workspace_bytes(N)) return GBCONV_ERR_WORKSPACE;
    return launch_nll_fwd(logp, target, weight, N, C, ignore_index, reduction, out, total_weight,
                          static_cast<float *>(ws), static_cast<cudaStream_t>(stream));
}

gbconv_status_t gbconv_nll_loss_bwd(const float *grad_out, const int64_t *target,
                                    const float *weight, int64_t N, int64_t C,
                                    int64_t ignore_index, int32_t reduction,
                                    const float *total_weight, float *grad_in,
                                    gbconv_stream_t stream) {
    if (N < 0 || C < 1 || reduction < 0 || reduction > 2) return GBCONV_ERR_INVALID_ARG;
    if (N == 0) return GBCONV_OK;
    if (!grad_out || !target || !grad_in || (reduction == 1 && !total_weight))
        return GBCONV_ERR_INVALID_ARG;
    if (N * C >= (1ll << 40)) return GBCONV_ERR_INVALID_ARG;
    return launch_nll_grad(grad_out, target, weight, N, C, ignore_index, reduction, total_weight,
                           grad_in, static_cast<cudaStream_t>(stream));
}

gbconv_status_t gbconv_bn_fold(int32_t K, const float *gamma, const float *bn_beta,
                               const float *mean, const float *var, float eps, const float *bias,
                               float *scale, float *shift, gbconv_stream_t stream) {
    if (K < 0) return GBCONV_ERR_INVALID_ARG;
    if (K == 0) return GBCONV_OK;
    if (!gamma || !bn_beta || !mean || !var || !scale || !shift || !(eps >= 0.f))
        return GBCONV_ERR_INVALID_ARG;
    return launch_bn_fold(K, gamma, bn_beta, mean, var, eps, bias, scale, shift,
                          static_cast<cudaStream_t>(stream));
}

gbconv_status_t conv2d_dgrad(const gbconv_problem_t *prob, const void *dy, const void *w,
                             void *dx, void *ws, size_t ws_bytes, gbconv_stream_t stream) {
    Dims d;
    gbconv_status_t s = make_dims(prob, &d);
    if (s != GBCONV_OK) return s;
    if (d.N == 0) return GBCONV_OK;  // empty batch: dx is empty
    if (!dy || !w || !dx || dx == dy || dx == w) return GBCONV_ERR_INVALID_ARG;
    const TcConfig c = config_for(GBCONV_OP_DGRAD, *prob, d);
    s = do_dgrad(d, c, dy, w, dx, ws, ws_bytes, static_cast<cudaStream_t>(stream));
    log_call("conv2d_dgrad", prob, &c, s);
    return s;
}

gbconv_status_t conv2d_wgrad(const gbconv_problem_t *prob, const void *x, const void *dy,
                             float *dw, float *db, void *ws, size_t ws_bytes,
                             gbconv_stream_t stream) {
    Dims d;
    gbconv_status_t s = make_dims(prob, &d);
    if (s != GBCONV_OK) return s;
    if (!dw || (d.N > 0 && (!x || !dy))) return GBCONV_ERR_INVALID_ARG;
    const TcConfig c = config_for(GBCONV_OP_WGRAD, *prob, d);
    s = do_wgrad(d, c, x, dy, dw, db, ws, ws_bytes, static_cast<cudaStream_t>(stream));
    log_call("conv2d_wgrad", prob, &c, s);
    return s;
}

gbconv_status_t conv2d_grouped(int32_t count, const gbconv_problem_t *probs, const void *const *x,
                               const void *const *w, const float *const *bias, void *const *y,
                               void *ws, size_t ws_bytes, gbconv_stream_t stream) {
    (void)ws;
    (void)ws_bytes;
    if (count < 0 || (count > 0 && (!probs || !x || !w || !y))) return GBCONV_ERR_INVALID_ARG;
    if (count == 0) return GBCONV_OK;
    std::vector<Dims> d(count);
    std::vector<TcConfig> cfg(count);
    std::vector<const float *> b(count);
    for (int i = 0; i < count; ++i) {
        gbconv_status_t s = make_dims(&probs[i], &d[i]);
        if (s != GBCONV_OK) return s;
        if (d[i].G > 1) return GBCONV_ERR_UNSUPPORTED;
        if (d[i].in_dtype != GBCONV_BF16 || d[i].out_dtype != GBCONV_BF16 ||
            d[i].layout != GBCONV_NHWC)
            return GBCONV_ERR_UNSUPPORTED;
        if (!x[i] || !w[i] || !y[i]) return GBCONV_ERR_INVALID_ARG;
        b[i] = bias ? bias[i] : nullptr;
        if ((d[i].flags & GBCONV_FLAG_BIAS) && !b[i]) return GBCONV_ERR_INVALID_ARG;
        s = check_tc_fwd(d[i], x[i], w[i], y[i]);
        if (s != GBCONV_OK) return s;
        cfg[i] = config_for(GBCONV_OP_GROUPED, probs[i], d[i]);
    }
    if (make_guard().err == nullptr) return GBCONV_ERR_CUDA;
    return launch_tc_grouped(count, d.data(), cfg.data(), x, w, b.data(), y,
                             static_cast<cudaStream_t>(stream));
}

gbconv_status_t gbconv_relu_grad(const void *y, int32_t y_dtype, const void *g, int32_t g_dtype,
                                 void *g_out, int32_t out_dtype, int64_t n, gbconv_stream_t stream) {
    if (n < 0) return GBCONV_ERR_INVALID_ARG;
    if (n == 0) return GBCONV_OK;
    if (!y || !g || !g_out) return GBCONV_ERR_INVALID_ARG;
    auto ok = [](int32_t t) { return t == GBCONV_F32 || t == GBCONV_BF16; };
    if (!ok(y_dtype) || !ok(g_dtype) || !ok(out_dtype)) return GBCONV_ERR_UNSUPPORTED;
    const int eo = out_dtype == GBCONV_F32 ? 4 : 2;
    const int eg = g_dtype == GBCONV_F32 ? 4 : 2;
    const int ey = y_dtype == GBCONV_F32 ? 4 : 2;
    // g_out may be g itself (same element type, same start) but must not
    // partly overlap g or overlap y at all
    auto overlap = [n](const void *a, int ea, const void *b, int eb) {
        const char *pa = static_cast<const char *>(a), *pb = static_cast<const char *>(b);
        return pa < pb + n * eb && pb < pa + n * ea;
    };
    if (overlap(g_out, eo, y, ey)) return GBCONV_ERR_INVALID_ARG;
    if (overlap(g_out, eo, g, eg) && !(g_out == g && eo == eg)) return GBCONV_ERR_INVALID_ARG;
    return launch_relu_grad(y, y_dtype, g, g_dtype, g_out, out_dtype, n,
                            static_cast<cudaStream_t>(stream));
}

gbconv_status_t gbconv_quantize_e4m3(const void *in, int32_t in_dtype, int64_t rows, int64_t len,
                                     uint8_t *out, float *scale, gbconv_stream_t stream) {
    if (!in || !out || !scale || rows < 1 || len < 1) return GBCONV_ERR_INVALID_ARG;
    if (in_dtype != GBCONV_F32 && in_dtype != GBCONV_BF16) return GBCONV_ERR_UNSUPPORTED;
    return launch_quantize_e4m3(in, in_dtype, rows, len, out, scale,
                                static_cast<cudaStream_t>(stream));
}

gbconv_status_t gbconv_get_config(int32_t op, const gbconv_problem_t *prob, gbconv_config_t *cfg) {
    Dims d;
    gbconv_status_t s = make_dims(prob, &d);
    if (s != GBCONV_OK) return s;
    if (!cfg || op < GBCONV_OP_FWD || op > GBCONV_OP_GROUPED) return GBCONV_ERR_INVALID_ARG;
    TcConfig c = config_for(op, *prob, d);
    cfg->block_n = c.block_n;
    cfg->stages = c.stages;
    cfg->split_k = c.split_k;
    cfg->raster = c.raster;
    cfg->algo = c.algo;
    return GBCONV_OK;
}

gbconv_status_t gbconv_set_config(int32_t op, const gbconv_problem_t *prob,
                                  const gbconv_config_t *cfg) {
    Dims d;
    gbconv_status_t s = make_dims(prob, &d);
    if (s != GBCONV_OK) return s;
    if (!cfg || op < GBCONV_OP_FWD || op > GBCONV_OP_GROUPED) return GBCONV_ERR_INVALID_ARG;
    if (cfg->block_n && cfg->block_n != 32 && cfg->block_n != 64 && cfg->block_n != 128 &&
        cfg->block_n != 256)
        return GBCONV_ERR_INVALID_ARG;
    if (cfg->split_k < 0 || cfg->split_k > 1024 || cfg->stages < 0 || cfg->raster < 0 ||
        cfg->raster > 1 || cfg->algo < GBCONV_ALGO_AUTO || cfg->algo > GBCONV_ALGO_PBAND_PAIR)
        return GBCONV_ERR_INVALID_ARG;
    TcConfig c = config_for(op, *prob, d);  // defaults for zero fields
    if (cfg->block_n) c.block_n = cfg->block_n;
    if (cfg->stages) c.stages = cfg->stages;
    if (cfg->split_k) c.split_k = cfg->split_k;
    // the band weight-gradient kernel's own default slice count
    else if (op == GBCONV_OP_WGRAD && cfg->algo == GBCONV_ALGO_SHIFT && tc_wgrad_shift_supported(d))
        c.split_k = tc_wgrad_shift_default_slices(d);
    c.raster = cfg->raster;
    c.algo = cfg->algo;
    std::string k = problem_key(op, *prob);
    std::lock_guard<std::mutex> lock(g_mu);
    g_tune[k] = c;
    return GBCONV_OK;
}

gbconv_status_t gbconv_tune(int32_t op, const gbconv_problem_t *prob, const void *a, const void *b,
                            const float *bias, void *out, void *ws, size_t ws_bytes, int32_t reps,
                            gbconv_stream_t stream, gbconv_config_t *best) {
    Dims d;
    gbconv_status_t s = make_dims(prob, &d);
    if (s != GBCONV_OK) return s;
    if (!a || !b || !out || op < GBCONV_OP_FWD || op > GBCONV_OP_GROUPED) return GBCONV_ERR_INVALID_ARG;
    if (d.G > 1) return GBCONV_ERR_UNSUPPORTED;  // grouped layers have no tunable configuration
    if (reps < 1) reps = 1;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const TcConfig base = config_for(op, *prob, d);
    std::vector<TcConfig> cands;
    if (op == GBCONV_OP_WGRAD) {
        // the per-tap kernel and the band kernel, each at a range of slice
        // counts including its default
        std::vector<int> algos;
        if (tc_wgrad_supported(d)) algos.push_back(GBCONV_ALGO_IM2COL);
        if (tc_wgrad_shift_supported(d)) algos.push_back(GBCONV_ALGO_SHIFT);
        if (algos.empty()) algos.push_back(base.algo);
        for (int algo : algos) {
            std::vector<int> splits = {1, 2, 4, 8, 16, 32, 64};
            if (algo == GBCONV_ALGO_SHIFT) splits.push_back(tc_wgrad_shift_default_slices(d));
            if (algo == GBCONV_ALGO_IM2COL) splits.push_back(tc_wgrad_default_config(d).split_k);
            std::sort(splits.begin(), splits.end());
            splits.erase(std::unique(splits.begin(), splits.end()), splits.end());
            for (int sk : splits) {
                TcConfig c = base;
                c.algo = algo;
                c.split_k = sk;
                if (wgrad_ws_bytes(d, sk) <= ws_bytes) cands.push_back(c);
            }
        }
    } else if (op == GBCONV_OP_GROUPED) {
        // the grouped launch's body (the im2col kernel): its per-problem tile width
        if (d.in_dtype != GBCONV_BF16 || d.out_dtype != GBCONV_BF16 || d.layout != GBCONV_NHWC ||
            check_tc_fwd(d, a, b, out) != GBCONV_OK)
            return GBCONV_ERR_UNSUPPORTED;
        for (int bn : {32, 64, 128, 256}) {
            if (bn > 32 && bn / 2 >= d.K) continue;
            TcConfig c = base;
            c.block_n = bn;
            c.algo = GBCONV_ALGO_IM2COL;
            cands.push_back(c);
        }
    } else {
        Dims t = d;
        const bool fwd_tc = op == GBCONV_OP_FWD && tc_fwd_supported(d);
        const bool rotated = op == GBCONV_OP_DGRAD && dgrad_as_fwd(d, &t);
        const bool phases = op == GBCONV_OP_DGRAD && !rotated && tc_dgrad_t_supported(d);
        const int kout = op == GBCONV_OP_FWD ? d.K : d.C;
        if (fwd_tc || rotated) {
            for (int bn : {32, 64, 128, 256}) {
                if (bn > 32 && bn / 2 >= kout) continue;  // wider than needed
                for (int algo : {GBCONV_ALGO_IM2COL, GBCONV_ALGO_SHIFT, GBCONV_ALGO_SHIFT_T}) {
                    if (algo == GBCONV_ALGO_SHIFT && !tc_fwd_shift_supported(t, bn)) continue;
                    // the transposed kernel picks its own tile: try it once
                    if (algo == GBCONV_ALGO_SHIFT_T && (!tc_fwd_t_tile(t) || bn != 64)) continue;
                    // the im2col ring depth is a launch parameter (0: the most that
                    // fits); the band kernels size their rings from the layer
                    const std::vector<int> stage_set = algo == GBCONV_ALGO_IM2COL
                                                           ? std::vector<int>{0, 4, 3}
                                                           : std::vector<int>{0};
                    for (int stages : stage_set)
                        for (int raster : {0, 1}) {
                            TcConfig c = base;
                            c.block_n = bn;
                            c.stages = stages;
                            c.raster = raster;
                            c.algo = algo;
                            cands.push_back(c);
                        }
                }
            }
            // the pixel-major band kernel picks its own tile: one SM, or a pair
            for (int form : {1, 2})
                if (tc_fwd_p_form(t, form) == form) {
                    TcConfig c = base;
                    c.algo = form == 1 ? GBCONV_ALGO_PBAND : GBCONV_ALGO_PBAND_PAIR;
                    cands.push_back(c);
                }
        } else if (phases) {
            // sub-pixel phases on the tensor cores, or the CUDA-core gather kernel
            for (int algo : {GBCONV_ALGO_AUTO, GBCONV_ALGO_SIMT}) {
                TcConfig c = base;
                c.algo = algo;
                cands.push_back(c);
            }
        } else {
            cands.push_back(base);
        }
    }
    if (cands.empty()) return GBCONV_ERR_WORKSPACE;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return GBCONV_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return GBCONV_ERR_CUDA;
    }
    float best_ms = 1e30f;
    TcConfig best_c = base;
    for (const TcConfig &c : cands) {
        auto run = [&]() -> gbconv_status_t {
            if (op == GBCONV_OP_FWD) return do_fwd(d, c, a, b, bias, nullptr, nullptr, out, st);
            if (op == GBCONV_OP_DGRAD) return do_dgrad(d, c, a, b, out, ws, ws_bytes, st);
            if (op == GBCONV_OP_GROUPED) {
                const void *xa[1] = {a}, *wb[1] = {b};
                const float *bb[1] = {(d.flags & GBCONV_FLAG_BIAS) ? bias : nullptr};
                void *ya[1] = {out};
                return launch_tc_grouped(1, &d, &c, xa, wb, bb, ya, st);
            }
            return do_wgrad(d, c, a, b, static_cast<float *>(out), nullptr, ws, ws_bytes, st);
        };
        if (run() != GBCONV_OK) continue;  // warm-up; skips configs that do not apply
        cudaEventRecord(e0, st);
        bool ok = true;
        for (int i = 0; i < reps && ok; ++i) ok = run() == GBCONV_OK;
        cudaEventRecord(e1, st);
        if (!ok || cudaEventSynchronize(e1) != cudaSuccess) continue;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
            best_ms = ms;
            best_c = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    {
        std::string k = problem_key(op, *prob);
        std::lock_guard<std::mutex> lock(g_mu);
        g_tune[k] = best_c;
    }
    {
        const char *path = getenv("GBCONV_TUNE_CACHE");
        if (path && *path) gbconv_tune_cache_save(path);
    }
    if (best) {
        best->block_n = best_c.block_n;
        best->stages = best_c.stages;
        best->split_k = best_c.split_k;
        best->raster = best_c.raster;
        best->algo = best_c.algo;
    }
    return gbconv_get_device_error(stream);
}

gbconv_status_t gbconv_tune_cache_save(const char *path) {
    if (!path) return GBCONV_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_mu);
    FILE *f = fopen(path, "w");
    if (!f) return GBCONV_ERR_INVALID_ARG;
    fprintf(f, "{\"version\": %d, \"entries\": [\n", 10000);
    bool first = true;
    for (auto &kv : g_tune) {
        fprintf(f,
                "%s {\"key\": \"%s\", \"block_n\": %d, \"stages\": %d, \"split_k\": %d, "
                "\"raster\": %d, \"algo\": %d}",
                first ? "" : ",\n", kv.first.c_str(), kv.second.block_n, kv.second.stages,
                kv.second.split_k, kv.second.raster, kv.second.algo);
        first = false;
    }
    fprintf(f, "\n]}\n");
    fclose(f);
    return GBCONV_OK;
}

gbconv_status_t gbconv_tune_cache_load(const char *path) {
    load_env_cache_once();  // an explicit load takes precedence over the environment's
    return gbc::load_cache_file(path);
}

}  // extern "C"

// Reads the format gbconv_tune_cache_save writes: one entry object per line.
gbconv_status_t gbc::load_cache_file(const char *path) {
    if (!path) return GBCONV_ERR_INVALID_ARG;
    FILE *f = fopen(path, "r");
    if (!f) return GBCONV_ERR_INVALID_ARG;
    char line[1024];
    std::map<std::string, TcConfig> add;
    while (fgets(line, sizeof line, f)) {
        const char *k = strstr(line, "\"key\": \"");
        if (!k) continue;
        k += 8;
        const char *ke = strchr(k, '"');
        if (!ke) continue;
        TcConfig c{};
        if (sscanf(ke,
                   "\", \"block_n\": %d, \"stages\": %d, \"split_k\": %d, \"raster\": %d, "
                   "\"algo\": %d",
                   &c.block_n, &c.stages, &c.split_k, &c.raster, &c.algo) != 5) {
            fclose(f);
            return GBCONV_ERR_INVALID_ARG;
        }
        add[std::string(k, ke)] = c;
    }
    fclose(f);
    std::lock_guard<std::mutex> lock(g_mu);
    for (auto &kv : add) g_tune[kv.first] = kv.second;
    return GBCONV_OK;
}

extern "C" {

gbconv_status_t gbconv_get_device_error(gbconv_stream_t stream) {
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess)
        return GBCONV_ERR_CUDA;
    DevInfo *di = dev_info();
    if (!di) return GBCONV_ERR_CUDA;
    unsigned int h = 0;
    if (cudaMemcpy(&h, di->err, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess)
        return GBCONV_ERR_CUDA;
    if (h != 0) {
        unsigned int z = 0;
        if (cudaMemcpy(di->err, &z, sizeof z, cudaMemcpyHostToDevice) != cudaSuccess)
            return GBCONV_ERR_CUDA;
        return (h & DEVERR_TIMEOUT) ? GBCONV_ERR_TIMEOUT : GBCONV_ERR_INVALID_ARG;
    }
    return GBCONV_OK;
}

const char *gbconv_status_string(gbconv_status_t s) {
    switch (s) {
        case GBCONV_OK: return "GBCONV_OK";
        case GBCONV_ERR_INVALID_ARG: return "GBCONV_ERR_INVALID_ARG";
        case GBCONV_ERR_UNSUPPORTED: return "GBCONV_ERR_UNSUPPORTED";
        case GBCONV_ERR_ALIGNMENT: return "GBCONV_ERR_ALIGNMENT";
        case GBCONV_ERR_WORKSPACE: return "GBCONV_ERR_WORKSPACE";
        case GBCONV_ERR_CUDA: return "GBCONV_ERR_CUDA";
        case GBCONV_ERR_TIMEOUT: return "GBCONV_ERR_TIMEOUT";
    }
    return "GBCONV_UNKNOWN_STATUS";
}

gbconv_status_t gbconv_debug_set(int32_t key, int64_t value) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (key == GBCONV_DEBUG_WAIT_LIMIT_NS) {
        if (value < 0) return GBCONV_ERR_INVALID_ARG;
        g_wait_ns = value == 0 ? default_wait_ns() : (uint64_t)value;
        return GBCONV_OK;
    }
    if (key == GBCONV_DEBUG_SKIP_LOADS) {
        g_skip_loads = value ? 1 : 0;
        return GBCONV_OK;
    }
    return GBCONV_ERR_INVALID_ARG;
}

// Device address of g_dgrad_static_scratch on the current device. In host
// code the array's name is only a host-side stand-in, so the real address is
// looked up once per device (with that device current) and cached.
static gbconv_status_t dgrad_static_scratch(void **out) {
    static std::mutex mu;
    static void *addr[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return GBCONV_ERR_CUDA;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_dgrad_static_scratch) != cudaSuccess || !p)
            return GBCONV_ERR_CUDA;
        addr[dev] = p;
    }
    *out = addr[dev];
    return GBCONV_OK;
}

gbconv_status_t conv2d_dgrad_noalloc(const gbconv_problem_t *prob, const void *dy, const void *w,
                                     void *dx, gbconv_stream_t stream) {
    Dims d;
    gbconv_status_t s = make_dims(prob, &d);
    if (s != GBCONV_OK) return s;
    if (d.N == 0) return GBCONV_OK;
    if (!dy || !w || !dx || dx == dy || dx == w) return GBCONV_ERR_INVALID_ARG;
    if (d.in_dtype == GBCONV_E4M3 || d.out_dtype == GBCONV_E4M3) return GBCONV_ERR_UNSUPPORTED;
    if (d.G > 1) return launch_simt_dgrad(d, dy, w, dx, static_cast<cudaStream_t>(stream));
    if (d.in_dtype == GBCONV_F32 && d.out_dtype != GBCONV_F32) return GBCONV_ERR_UNSUPPORTED;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const TcConfig cfg = config_for(GBCONV_OP_DGRAD, *prob, d);
    Dims t;
    const bool rotated = cfg.algo != GBCONV_ALGO_SIMT && dgrad_as_fwd(d, &t);
    const bool phases = cfg.algo != GBCONV_ALGO_SIMT && !rotated && tc_dgrad_t_supported(d);
    if (!rotated && !phases) return launch_simt_dgrad(d, dy, w, dx, st);  // no scratch used
    // the tensor-core forms keep the filter, rotated (stride 1) or transposed
    // (sub-pixel phases of strided layers), in the static scratch
    const size_t need = (size_t)d.K * d.R * d.S * d.C * 2;
    if (need > (size_t)GBCONV_DGRAD_STATIC_SCRATCH_BYTES) return GBCONV_ERR_WORKSPACE;
    if (!aligned16(dy) || !aligned16(dx)) return GBCONV_ERR_ALIGNMENT;
    void *scratch = nullptr;
    s = dgrad_static_scratch(&scratch);
    if (s != GBCONV_OK) return s;
    if (phases) {
        s = launch_transpose_filter(d, w, scratch, st);
        if (s != GBCONV_OK) return s;
        return launch_tc_dgrad_t(d, dy, scratch, dx, st);
    }
    s = launch_rotate_filter(d, w, scratch, st);
    if (s != GBCONV_OK) return s;
    return launch_tc_fwd(t, cfg, dy, scratch, nullptr, nullptr, nullptr, dx, st);
}

gbconv_status_t gbconv_measure_ffma_tflops(int64_t iters, double *tflops, gbconv_stream_t stream) {
    if (iters < 1 || !tflops) return GBCONV_ERR_INVALID_ARG;
    return measure_ffma_rate(iters, tflops, static_cast<cudaStream_t>(stream));
}

int32_t gbconv_version(void) { return 10000; }

void gbconv_shutdown(void) {
    std::lock_guard<std::mutex> lock(g_mu);
    g_tune.clear();
}

}  // extern "C"
