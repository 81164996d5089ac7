/*
 * All-core timing of the oracle's two embarrassingly parallel stages: the
 * crossed-face set C (Alg. 3's face loop with Alg. 1) and the verification
 * of a reconstruction (Eq. 4 on every face, plus the pointwise bound).
 *
 * TEST AND BENCHMARK INFRASTRUCTURE ONLY, like the oracle itself: only the
 * tests and the CPU-baseline leg of the benchmark load this library.
 *
 * Nothing here changes the oracle's arithmetic: this file includes the
 * oracle's source unchanged and runs its own o_face_masks on two-slice slabs
 * [t, t+1], one slab at a time per host thread.  The masks of slice t are a
 * function of slices t and t+1 only, and the symbolic perturbation orders a
 * face's vertices by their relative offsets, which a slab keeps; so slab t
 * gives slice t's masks exactly as the whole field does.
 */
#include <pthread.h>
#include <stdatomic.h>

#include "cpt_oracle.c"

typedef struct {
    const int32_t* q;      /* field whose masks are computed */
    const uint16_t* ref;   /* NULL: store masks; else compare against them */
    const float* uv;       /* verification: the original values */
    uint16_t* mask;        /* out (mask mode) */
    int H, W, T, k;
    atomic_int next;       /* next slice to take */
    int err;
    /* verification totals, per thread then summed */
    u64 mism_slice[256], mism_slab[256];
    double linf[256];
} par_job;

typedef struct {
    par_job* job;
    int id;
} par_arg;

static void* par_worker(void* p) {
    par_arg* a = (par_arg*)p;
    par_job* J = a->job;
    const i64 sl = (i64)J->H * J->W;
    uint16_t* buf = (uint16_t*)malloc(sizeof(uint16_t) * 2 * (size_t)sl);
    if (!buf) {
        J->err = O_ERR_OOM;
        return NULL;
    }
    u64 ms = 0, mb = 0;
    double linf = 0.0;
    for (;;) {
        int t = atomic_fetch_add(&J->next, 1);
        if (t >= J->T) break;
        const int nt = t + 1 < J->T ? 2 : 1;
        o_face_masks(J->q + 2 * sl * t, J->H, J->W, nt, buf);
        if (!J->ref) {
            memcpy(J->mask + sl * t, buf, sizeof(uint16_t) * (size_t)sl);
            continue;
        }
        const uint16_t* r = J->ref + sl * t;
        for (i64 v = 0; v < sl; ++v) {
            unsigned x = (unsigned)(buf[v] ^ r[v]);
            for (int b = 0; b < 12; ++b)
                if ((x >> b) & 1u) {
                    if (b < 2) ++ms;
                    else ++mb;
                }
        }
        /* x_hat = q_hat * 2^-k exactly; |x_hat - x| in double */
        const i64 base = 2 * sl * t;
        for (i64 n = 0; n < 2 * sl; ++n) {
            double e = fabs(ldexp((double)J->q[base + n], -J->k) - (double)J->uv[base + n]);
            if (e > linf) linf = e;
        }
    }
    free(buf);
    J->mism_slice[a->id] = ms;
    J->mism_slab[a->id] = mb;
    J->linf[a->id] = linf;
    return NULL;
}

static int par_run(par_job* J, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    par_arg args[256];
    atomic_init(&J->next, 0);
    J->err = 0;
    int started = 0;
    for (int i = 0; i < nthreads; ++i) {
        args[i].job = J;
        args[i].id = i;
        J->mism_slice[i] = J->mism_slab[i] = 0;
        J->linf[i] = 0.0;
        if (pthread_create(&th[i], NULL, par_worker, &args[i]) != 0) break;
        ++started;
    }
    if (started == 0) return O_ERR_OOM;
    for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
    return J->err;
}

/* C as 12-bit masks per owner vertex, like o_face_masks, on nthreads threads. */
int o_face_masks_par(const int32_t* q, int H, int W, int T, uint16_t* mask, int nthreads) {
    par_job* J = (par_job*)calloc(1, sizeof(par_job));
    if (!J) return O_ERR_OOM;
    J->q = q;
    J->mask = mask;
    J->H = H;
    J->W = W;
    J->T = T;
    int rc = par_run(J, nthreads);
    free(J);
    return rc;
}

/* Verification of a reconstruction q_hat (fixed point, exponent k) against
 * the original's masks and values: face predicates that differ (slice faces
 * and slab faces counted apart) and the largest pointwise error. */
int o_verify_par(const int32_t* qhat, const uint16_t* mask, const float* uv, int H, int W, int T, int k,
                 int nthreads, u64* mism_slice, u64* mism_slab, double* linf) {
    par_job* J = (par_job*)calloc(1, sizeof(par_job));
    if (!J) return O_ERR_OOM;
    J->q = qhat;
    J->ref = mask;
    J->uv = uv;
    J->H = H;
    J->W = W;
    J->T = T;
    J->k = k;
    int rc = par_run(J, nthreads);
    u64 a = 0, b = 0;
    double l = 0.0;
    for (int i = 0; i < 256; ++i) {
        a += J->mism_slice[i];
        b += J->mism_slab[i];
        if (J->linf[i] > l) l = J->linf[i];
    }
    *mism_slice = a;
    *mism_slab = b;
    *linf = l;
    free(J);
    return rc;
}
