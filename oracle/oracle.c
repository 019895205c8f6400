/*
 * oracle.c -- plain FP64 CPU oracle for dense 2D convolution.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may link, load or
 * call this file: only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline leg use it. It shares no code, header, table or helper with the
 * CUDA library under paper_2207_00257_gb300/csrc/.
 *
 * What it computes (paper, Sec. 1 and Sec. 5.A: the PyTorch native CPU
 * backend runs 2D convolution as six nested loops; Sec. 5.B: the forward and
 * backward passes of the convolutional layers, NCHW layout):
 *
 *   y[n,k,p,q] = b[k] + sum_{c<C, r<R, s<S} x[n,c, p*u + r*dh - ph,
 *                                               q*v + s*dw - pw] * w[k,c,r,s]
 *
 * with out-of-range x taken as 0, P = floor((H + 2ph - dh(R-1) - 1)/u) + 1 and
 * Q likewise (cross-correlation, no filter flip). For the loss L = sum g*y:
 *
 *   dx[n,c,h,w] = sum over (k,r,s,p,q) with p*u + r*dh - ph = h and
 *                 q*v + s*dw - pw = w of g[n,k,p,q] * w[k,c,r,s]
 *   dw[k,c,r,s] = sum_{n,p,q} g[n,k,p,q] * x[n,c,p*u+r*dh-ph,q*v+s*dw-pw]
 *   db[k]       = sum_{n,p,q} g[n,k,p,q]
 *
 * The layers around a ResNet-50 convolution (Sec. 5.B: batch normalisation
 * and tensor additions follow the convolutions) give the fused forward
 *
 *   y[n,k,p,q] = act(alpha[k] * conv[n,k,p,q] + beta[k] + z[n,k,p,q])
 *
 * (conv the sum above without bias, alpha a per-channel scale, beta a
 * per-channel shift, z a residual tensor of y's shape, act ReLU or identity),
 * and inference batch normalisation folded into (alpha, beta):
 *
 *   alpha[k] = gamma[k] / sqrt(var[k] + eps)
 *   beta[k]  = bn_beta[k] + (b[k] - mean[k]) * alpha[k]
 *
 * so that alpha*(conv + b) normalised by (mean, var) and shifted by bn_beta
 * equals alpha*conv + beta.
 *
 * Every function here is the definition written out as loops in double
 * precision, with the loop order n,k,p,q outside and c,r,s inside. There is
 * no blocking, no im2col and no reordering of the sum. Threads only split the
 * set of outputs; each output is still one serial double-precision sum.
 *
 * Layouts: layout 0 = NCHW activations with KCRS filters; layout 1 = NHWC
 * activations with KRSC filters. Output y / gradient g follow the activation
 * layout (NKPQ or NPQK).
 *
 * Quantisers: FP32 -> BF16 round-to-nearest-even, and FP32 -> FP8 E4M3
 * (OCP 8-bit floating point, E4M3 variant: bias 7, no infinities, only
 * S.1111.111 is NaN, largest finite 448) round-to-nearest-even with
 * saturation to +-448. Both are written from those format definitions.
 *
 * Channel groups (G = groups; G = C = K is the depthwise convolution): the
 * C input and K output channels split into G equal groups, output channel k
 * of group g = k / (K/G) reads only input channels g*(C/G) .. g*(C/G)+C/G-1,
 * and the filter holds C/G channels per output channel:
 *
 *   y[n,k,p,q] = b[k] + sum_{c<C/G, r, s} x[n, g*(C/G) + c, ...] * w[k,c,r,s]
 *
 * (the data and weight gradients restrict their sums the same way).
 *
 * Dims are passed as int64 d[15] = {N,C,H,W,K,R,S,u,v,ph,pw,dh,dw,layout,G}.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

typedef struct {
    int64_t N, C, H, W, K, R, S, u, v, ph, pw, dh, dw, layout, P, Q;
    int64_t G, Cg, Kg;  /* groups, input and output channels per group */
} dims_t;

static int load_dims(const int64_t *d, dims_t *o) {
    o->N = d[0]; o->C = d[1]; o->H = d[2]; o->W = d[3]; o->K = d[4];
    o->R = d[5]; o->S = d[6]; o->u = d[7]; o->v = d[8]; o->ph = d[9];
    o->pw = d[10]; o->dh = d[11]; o->dw = d[12]; o->layout = d[13]; o->G = d[14];
    if (o->N < 0 || o->C < 1 || o->H < 1 || o->W < 1 || o->K < 1 || o->R < 1 ||
        o->S < 1 || o->u < 1 || o->v < 1 || o->ph < 0 || o->pw < 0 ||
        o->dh < 1 || o->dw < 1 || (o->layout != 0 && o->layout != 1) || o->G < 1 ||
        o->C % o->G != 0 || o->K % o->G != 0)
        return -1;
    o->Cg = o->C / o->G;
    o->Kg = o->K / o->G;
    int64_t pn = o->H + 2 * o->ph - o->dh * (o->R - 1) - 1;
    int64_t qn = o->W + 2 * o->pw - o->dw * (o->S - 1) - 1;
    if (pn < 0 || qn < 0) return -1;
    o->P = pn / o->u + 1;
    o->Q = qn / o->v + 1;
    return 0;
}

/* Output size, as the PyTorch formula above. Returns -1 on invalid dims. */
int oracle_output_dims(const int64_t *d, int64_t *P, int64_t *Q) {
    dims_t D;
    if (load_dims(d, &D)) return -1;
    *P = D.P; *Q = D.Q;
    return 0;
}

static inline int64_t xi(const dims_t *D, int64_t n, int64_t c, int64_t h, int64_t w) {
    return D->layout == 0 ? ((n * D->C + c) * D->H + h) * D->W + w
                          : ((n * D->H + h) * D->W + w) * D->C + c;
}
/* filter element (k, c, r, s), c < C/G the channel within k's group */
static inline int64_t wi(const dims_t *D, int64_t k, int64_t c, int64_t r, int64_t s) {
    return D->layout == 0 ? ((k * D->Cg + c) * D->R + r) * D->S + s
                          : ((k * D->R + r) * D->S + s) * D->Cg + c;
}
static inline int64_t yi(const dims_t *D, int64_t n, int64_t k, int64_t p, int64_t q) {
    return D->layout == 0 ? ((n * D->K + k) * D->P + p) * D->Q + q
                          : ((n * D->P + p) * D->Q + q) * D->K + k;
}
/* Inverse of yi / xi / wi: linear index -> coordinates. */
static void y_coords(const dims_t *D, int64_t i, int64_t *n, int64_t *k, int64_t *p, int64_t *q) {
    if (D->layout == 0) {
        *q = i % D->Q; i /= D->Q; *p = i % D->P; i /= D->P; *k = i % D->K; *n = i / D->K;
    } else {
        *k = i % D->K; i /= D->K; *q = i % D->Q; i /= D->Q; *p = i % D->P; *n = i / D->P;
    }
}
static void x_coords(const dims_t *D, int64_t i, int64_t *n, int64_t *c, int64_t *h, int64_t *w) {
    if (D->layout == 0) {
        *w = i % D->W; i /= D->W; *h = i % D->H; i /= D->H; *c = i % D->C; *n = i / D->C;
    } else {
        *c = i % D->C; i /= D->C; *w = i % D->W; i /= D->W; *h = i % D->H; *n = i / D->H;
    }
}
static void w_coords(const dims_t *D, int64_t i, int64_t *k, int64_t *c, int64_t *r, int64_t *s) {
    if (D->layout == 0) {
        *s = i % D->S; i /= D->S; *r = i % D->R; i /= D->R; *c = i % D->Cg; *k = i / D->Cg;
    } else {
        *c = i % D->Cg; i /= D->Cg; *s = i % D->S; i /= D->S; *r = i % D->R; *k = i / D->R;
    }
}

/* ---- one output of each operation, straight from the definitions ---- */

/* y[n,k,p,q] (before the optional bias/ReLU) and its error normaliser
 * sum |x||w| over the same in-range terms. */
static void fwd_one(const dims_t *D, const double *x, const double *w, int64_t n,
                    int64_t k, int64_t p, int64_t q, double *sum, double *abssum) {
    double acc = 0.0, aacc = 0.0;
    const int64_t c0 = (k / D->Kg) * D->Cg;  /* first input channel of k's group */
    for (int64_t c = 0; c < D->Cg; ++c)
        for (int64_t r = 0; r < D->R; ++r)
            for (int64_t s = 0; s < D->S; ++s) {
                int64_t h = p * D->u + r * D->dh - D->ph;
                int64_t ww = q * D->v + s * D->dw - D->pw;
                if (h < 0 || h >= D->H || ww < 0 || ww >= D->W) continue;
                double a = x[xi(D, n, c0 + c, h, ww)], f = w[wi(D, k, c, r, s)];
                acc += a * f;
                aacc += fabs(a) * fabs(f);
            }
    *sum = acc;
    *abssum = aacc;
}

/* dx[n,c,h,w]: every (k,r,s,p,q) whose tap lands on (h,w). */
static void dgrad_one(const dims_t *D, const double *g, const double *w, int64_t n,
                      int64_t c, int64_t h, int64_t ww, double *sum, double *abssum) {
    double acc = 0.0, aacc = 0.0;
    const int64_t grp = c / D->Cg, cl = c - grp * D->Cg;  /* c's group, channel within it */
    for (int64_t k = grp * D->Kg; k < (grp + 1) * D->Kg; ++k)
        for (int64_t r = 0; r < D->R; ++r)
            for (int64_t s = 0; s < D->S; ++s) {
                int64_t pn = h + D->ph - r * D->dh;   /* = p*u */
                int64_t qn = ww + D->pw - s * D->dw;  /* = q*v */
                if (pn < 0 || qn < 0 || pn % D->u != 0 || qn % D->v != 0) continue;
                int64_t p = pn / D->u, q = qn / D->v;
                if (p >= D->P || q >= D->Q) continue;
                double a = g[yi(D, n, k, p, q)], f = w[wi(D, k, cl, r, s)];
                acc += a * f;
                aacc += fabs(a) * fabs(f);
            }
    *sum = acc;
    *abssum = aacc;
}

/* dw[k,c,r,s] = sum over n,p,q of g * x at the tap's input position (input
 * channel c of k's group). */
static void wgrad_one(const dims_t *D, const double *x, const double *g, int64_t k,
                      int64_t c, int64_t r, int64_t s, double *sum, double *abssum) {
    double acc = 0.0, aacc = 0.0;
    const int64_t cx = (k / D->Kg) * D->Cg + c;
    for (int64_t n = 0; n < D->N; ++n)
        for (int64_t p = 0; p < D->P; ++p)
            for (int64_t q = 0; q < D->Q; ++q) {
                int64_t h = p * D->u + r * D->dh - D->ph;
                int64_t ww = q * D->v + s * D->dw - D->pw;
                if (h < 0 || h >= D->H || ww < 0 || ww >= D->W) continue;
                double a = g[yi(D, n, k, p, q)], f = x[xi(D, n, cx, h, ww)];
                acc += a * f;
                aacc += fabs(a) * fabs(f);
            }
    *sum = acc;
    *abssum = aacc;
}

/* ---- a minimal parallel-for over independent outputs ---- */

typedef struct {
    const dims_t *D;
    const double *a, *b, *bias;
    const double *alpha, *z;  /* fused forward: per-channel scale, residual (may be NULL) */
    const int64_t *idx;   /* NULL: all outputs 0..count-1 */
    int64_t count;
    int op;               /* 0 fwd, 1 dgrad, 2 wgrad */
    int relu;
    double *out, *bound;  /* bound may be NULL */
    int tid, nthreads;
} job_t;

static void do_item(job_t *J, int64_t i) {
    const dims_t *D = J->D;
    int64_t lin = J->idx ? J->idx[i] : i;
    double sum = 0.0, asum = 0.0;
    if (J->op == 0) {
        int64_t n, k, p, q;
        y_coords(D, lin, &n, &k, &p, &q);
        fwd_one(D, J->a, J->b, n, k, p, q, &sum, &asum);
        if (J->alpha) {
            sum = J->alpha[k] * sum;
            asum = fabs(J->alpha[k]) * asum;
        }
        if (J->bias) {
            sum = J->bias[k] + sum;
            asum = fabs(J->bias[k]) + asum;
        }
        if (J->z) {
            sum = sum + J->z[lin];
            asum = asum + fabs(J->z[lin]);
        }
        if (J->relu && sum < 0.0) sum = 0.0;
    } else if (J->op == 1) {
        int64_t n, c, h, w;
        x_coords(D, lin, &n, &c, &h, &w);
        dgrad_one(D, J->a, J->b, n, c, h, w, &sum, &asum);
    } else {
        int64_t k, c, r, s;
        w_coords(D, lin, &k, &c, &r, &s);
        wgrad_one(D, J->a, J->b, k, c, r, s, &sum, &asum);
    }
    J->out[i] = sum;
    if (J->bound) J->bound[i] = asum;
}

static void *worker(void *arg) {
    job_t *J = (job_t *)arg;
    for (int64_t i = J->tid; i < J->count; i += J->nthreads) do_item(J, i);
    return NULL;
}

static int run(job_t proto, int nthreads) {
    if (nthreads <= 0) nthreads = (int)sysconf(_SC_NPROCESSORS_ONLN);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 512) nthreads = 512;
    if ((int64_t)nthreads > proto.count) nthreads = proto.count > 0 ? (int)proto.count : 1;
    job_t *jobs = (job_t *)calloc((size_t)nthreads, sizeof(job_t));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    char *live = (char *)calloc((size_t)nthreads, 1);
    if (!jobs || !th || !live) { free(jobs); free(th); free(live); return -2; }
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = proto;
        jobs[t].tid = t;
        jobs[t].nthreads = nthreads;
    }
    for (int t = 1; t < nthreads; ++t)
        live[t] = pthread_create(&th[t], NULL, worker, &jobs[t]) == 0;
    worker(&jobs[0]);
    for (int t = 1; t < nthreads; ++t) {
        if (live[t]) pthread_join(th[t], NULL);
        else worker(&jobs[t]);   /* thread could not start: do its share here */
    }
    free(jobs);
    free(th);
    free(live);
    return 0;
}

static int64_t y_count(const dims_t *D) { return D->N * D->K * D->P * D->Q; }
static int64_t x_count(const dims_t *D) { return D->N * D->C * D->H * D->W; }
static int64_t w_count(const dims_t *D) { return D->K * D->Cg * D->R * D->S; }

/* ---- exported entry points ---- */

/* Forward over all outputs (idx == NULL, npts ignored) or over the npts linear
 * output indices idx[]. bias may be NULL. relu != 0 applies max(0, .) after
 * the bias. bound (may be NULL) receives |b[k]| + sum |x||w|. */
int oracle_conv2d_fwd(const int64_t *d, const double *x, const double *w, const double *bias,
                      int relu, const int64_t *idx, int64_t npts, double *y, double *bound,
                      int nthreads) {
    dims_t D;
    if (load_dims(d, &D)) return -1;
    job_t J = {&D, x, w, bias, NULL, NULL, idx, idx ? npts : y_count(&D), 0, relu, y, bound, 0, 1};
    return run(J, nthreads);
}

/* Fused forward: y = act(alpha[k]*conv + beta[k] + z) at all outputs or at
 * the npts linear indices idx[]. alpha, beta, z may each be NULL (1, 0, 0); z
 * has y's shape and layout. bound receives |alpha[k]| sum |x||w| + |beta[k]|
 * + |z|. */
int oracle_conv2d_fwd_fused(const int64_t *d, const double *x, const double *w,
                            const double *alpha, const double *beta, const double *z, int relu,
                            const int64_t *idx, int64_t npts, double *y, double *bound,
                            int nthreads) {
    dims_t D;
    if (load_dims(d, &D)) return -1;
    job_t J = {&D, x, w, beta, alpha, z, idx, idx ? npts : y_count(&D), 0, relu, y, bound, 0, 1};
    return run(J, nthreads);
}

/* Inference batch normalisation folded into a per-channel scale and shift
 * (see the header); bias may be NULL (0). */
void oracle_bn_fold(int64_t K, const double *gamma, const double *bn_beta, const double *mean,
                    const double *var, double eps, const double *bias, double *alpha,
                    double *beta) {
    for (int64_t k = 0; k < K; ++k) {
        alpha[k] = gamma[k] / sqrt(var[k] + eps);
        beta[k] = bn_beta[k] + ((bias ? bias[k] : 0.0) - mean[k]) * alpha[k];
    }
}

/* dx over all inputs or at npts linear x indices. */
int oracle_conv2d_dgrad(const int64_t *d, const double *g, const double *w, const int64_t *idx,
                        int64_t npts, double *dx, double *bound, int nthreads) {
    dims_t D;
    if (load_dims(d, &D)) return -1;
    job_t J = {&D, g, w, NULL, NULL, NULL, idx, idx ? npts : x_count(&D), 1, 0, dx, bound, 0, 1};
    return run(J, nthreads);
}

/* dw over all filter taps or at npts linear w indices. */
int oracle_conv2d_wgrad(const int64_t *d, const double *x, const double *g, const int64_t *idx,
                        int64_t npts, double *dw, double *bound, int nthreads) {
    dims_t D;
    if (load_dims(d, &D)) return -1;
    job_t J = {&D, x, g, NULL, NULL, NULL, idx, idx ? npts : w_count(&D), 2, 0, dw, bound, 0, 1};
    return run(J, nthreads);
}

/* db[k] = sum_{n,p,q} g[n,k,p,q]; bound[k] = sum |g|. */
int oracle_conv2d_bgrad(const int64_t *d, const double *g, double *db, double *bound) {
    dims_t D;
    if (load_dims(d, &D)) return -1;
    for (int64_t k = 0; k < D.K; ++k) {
        double acc = 0.0, aacc = 0.0;
        for (int64_t n = 0; n < D.N; ++n)
            for (int64_t p = 0; p < D.P; ++p)
                for (int64_t q = 0; q < D.Q; ++q) {
                    double a = g[yi(&D, n, k, p, q)];
                    acc += a;
                    aacc += fabs(a);
                }
        db[k] = acc;
        if (bound) bound[k] = aacc;
    }
    return 0;
}

/* ---- quantisers ---- */

/* FP32 -> BF16, round to nearest, ties to even, on the upper 16 bits of the
 * binary32 pattern; NaN stays NaN (quiet bit forced); overflow rounds to inf
 * as RNE requires. */
void oracle_round_bf16(const float *in, uint16_t *out, int64_t n) {
    for (int64_t i = 0; i < n; ++i) {
        uint32_t b;
        memcpy(&b, &in[i], 4);
        if ((b & 0x7F800000u) == 0x7F800000u && (b & 0x007FFFFFu)) {
            out[i] = (uint16_t)((b >> 16) | 0x0040u);
            continue;
        }
        uint32_t keep = b >> 16, rest = b & 0xFFFFu;
        if (rest > 0x8000u || (rest == 0x8000u && (keep & 1u))) keep += 1u;
        out[i] = (uint16_t)keep;
    }
}

void oracle_bf16_to_f64(const uint16_t *in, double *out, int64_t n) {
    for (int64_t i = 0; i < n; ++i) {
        uint32_t b = (uint32_t)in[i] << 16;
        float f;
        memcpy(&f, &b, 4);
        out[i] = (double)f;
    }
}

/* Value of one E4M3 code. */
static double e4m3_value(uint8_t code) {
    int sign = code >> 7, e = (code >> 3) & 0xF, m = code & 7;
    if (e == 15 && m == 7) return NAN;
    double mag = (e == 0) ? ldexp((double)m, -9)               /* m/8 * 2^-6 */
                          : ldexp(8.0 + (double)m, e - 7 - 3); /* (1+m/8) 2^(e-7) */
    return sign ? -mag : mag;
}

void oracle_e4m3_to_f64(const uint8_t *in, double *out, int64_t n) {
    for (int64_t i = 0; i < n; ++i) out[i] = e4m3_value(in[i]);
}

/* Round |a| (finite, >= 0) to the E4M3 grid: the spacing is 2^(E-3) where E is
 * the binade exponent, and 2^-9 in the subnormal range (E < -6). Ties go to
 * the even grid point; values past 448 saturate to 448. */
static uint8_t e4m3_encode(double a) {
    if (a >= 448.0) return 0x7E;               /* S.1111.110 = 448 */
    if (a == 0.0) return 0;
    int E;
    (void)frexp(a, &E);                        /* a = f * 2^E, f in [0.5,1) */
    E -= 1;                                    /* a in [2^E, 2^(E+1)) */
    if (E < -6) E = -6;                        /* subnormal spacing */
    double quantum = ldexp(1.0, E - 3);
    double r = a / quantum;                    /* exact: power-of-two scale */
    double fl = floor(r), diff = r - fl;
    double m = fl;
    if (diff > 0.5 || (diff == 0.5 && fmod(fl, 2.0) != 0.0)) m = fl + 1.0;
    double v = m * quantum;
    if (v >= 448.0) return 0x7E;
    if (v == 0.0) return 0;
    int Ev;
    (void)frexp(v, &Ev);
    Ev -= 1;
    if (Ev < -6) return (uint8_t)ldexp(v, 9);  /* subnormal: mantissa = v / 2^-9 */
    int mant = (int)(ldexp(v, -Ev) * 8.0) - 8; /* v / 2^Ev = 1 + mant/8 */
    return (uint8_t)(((Ev + 7) << 3) | mant);
}

/* FP32 -> E4M3 with saturation; NaN -> 0x7F (sign kept). */
void oracle_quant_e4m3(const float *in, uint8_t *out, int64_t n) {
    for (int64_t i = 0; i < n; ++i) {
        float f = in[i];
        if (f != f) { out[i] = (uint8_t)(0x7F | (signbit(f) ? 0x80 : 0)); continue; }
        uint8_t mag = e4m3_encode(fabs((double)f));
        out[i] = (uint8_t)(mag | (signbit(f) ? 0x80 : 0));
    }
}

/* FP8 operand preparation (per-tensor or per-row scale), all in binary32:
 *   s = max|v| / 448 (with a floor so an all-zero tensor keeps s > 0),
 *   q = sat_E4M3(v / s) rounded to nearest even.
 * rows = number of independent scale groups, each of len contiguous values.
 * scales receives rows binary32 scales. */
void oracle_scale_quant_e4m3(const float *in, int64_t rows, int64_t len, uint8_t *out,
                             float *scales) {
    for (int64_t r = 0; r < rows; ++r) {
        const float *v = in + r * len;
        float amax = 0.0f;
        for (int64_t i = 0; i < len; ++i) {
            float a = fabsf(v[i]);
            if (a > amax) amax = a;
        }
        float s = amax / 448.0f;
        if (!(s >= 1.0e-12f)) s = 1.0e-12f;
        scales[r] = s;
        for (int64_t i = 0; i < len; ++i) {
            float t = v[i] / s;
            oracle_quant_e4m3(&t, out + r * len + i, 1);
        }
    }
}

/* ---- negative log-likelihood loss (Sec. 5.B: the ClassNLLCriterion forward
 * and gradient that ResNet-50 training calls after the network) ----
 *
 * logp is [N][C] (log-probabilities), target[n] a class index or ignore_index,
 * weight[c] an optional class weight (NULL: 1). With w_n = weight[target[n]]
 * for counted rows and 0 for ignored ones:
 *   reduction 0 (none): out[n] = -w_n * logp[n][target[n]]
 *   reduction 2 (sum):  out    = sum_n -w_n * logp[n][target[n]]
 *   reduction 1 (mean): out    = (sum_n -w_n * logp[n][target[n]]) / sum_n w_n
 * total_weight = sum_n w_n. The gradient with respect to logp for the
 * upstream gradient g (one value, or N values for reduction none) is zero
 * except at (n, target[n]) of counted rows: -w_n * g (none: g[n]; sum: g;
 * mean: g / total_weight). Returns -3 if a target is neither a class nor
 * ignore_index. */
int oracle_nll_loss_fwd(const double *logp, const int64_t *target, const double *weight,
                        int64_t N, int64_t C, int64_t ignore_index, int reduction, double *out,
                        double *total_weight) {
    double sum = 0.0, tw = 0.0;
    for (int64_t n = 0; n < N; ++n) {
        const int64_t t = target[n];
        if (t == ignore_index) {
            if (reduction == 0) out[n] = 0.0;
            continue;
        }
        if (t < 0 || t >= C) return -3;
        const double w = weight ? weight[t] : 1.0;
        const double v = -w * logp[n * C + t];
        if (reduction == 0) out[n] = v;
        sum += v;
        tw += w;
    }
    if (reduction == 1) out[0] = sum / tw;
    if (reduction == 2) out[0] = sum;
    *total_weight = tw;
    return 0;
}

int oracle_nll_loss_bwd(const double *grad_out, const int64_t *target, const double *weight,
                        int64_t N, int64_t C, int64_t ignore_index, int reduction,
                        double total_weight, double *grad_in) {
    for (int64_t i = 0; i < N * C; ++i) grad_in[i] = 0.0;
    for (int64_t n = 0; n < N; ++n) {
        const int64_t t = target[n];
        if (t == ignore_index) continue;
        if (t < 0 || t >= C) return -3;
        const double w = weight ? weight[t] : 1.0;
        const double g = reduction == 0 ? grad_out[n]
                         : reduction == 1 ? grad_out[0] / total_weight : grad_out[0];
        grad_in[n * C + t] = -w * g;
    }
    return 0;
}
