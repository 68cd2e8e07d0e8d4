// lse_reduce.cuh -- deterministic CTA/grid reductions and the per-iteration
// finalisation of the region statistics (internal).
//
// Every reducing kernel accumulates per thread, reduces its CTA in a fixed
// order (warp shuffles, then warps in index order), writes one LsePartial per
// CTA, and the last CTA to take a ticket sums the partials in CTA order and
// finalises.  The last CTA resets the ticket for the next launch.
#pragma once

#include "lse_internal.h"

struct LseAcc {
    double sp[LSE_MAXB];
    double sm[LSE_MAXB];
    long long n_plus;
    long long flips;
    float fmax, fmin;
    unsigned int bits;

    __device__ __forceinline__ void clear()
    {
#pragma unroll
        for (int b = 0; b < LSE_MAXB; ++b) {
            sp[b] = 0.0;
            sm[b] = 0.0;
        }
        n_plus = 0;
        flips = 0;
        fmax = -INFINITY;
        fmin = INFINITY;
        bits = 0;
    }
};

// Compensated summation (Kahan, 1965): s is the running FP32 sum and c the
// rounding error of its last addition, negated; the sum is s - c, within
// about 2 * 2^-24 of sum |x| however many terms are added.  The explicit
// round-to-nearest intrinsics keep the steps from being contracted or
// reassociated.  Per-pixel sums use it in place of FP64 additions, which
// this part issues at a small fraction of the FP32 rate.
__device__ __forceinline__ void lse_kahan_add(float &s, float &c, float x)
{
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

__device__ __forceinline__ double lse_kahan_value(float s, float c)
{
    return (double)s - (double)c;
}

// Knuth's TwoSum: s = fl(a + b) and e with s + e == a + b exactly.
__device__ __forceinline__ float lse_two_sum(float a, float b, float &e)
{
    const float s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    const float av = __fsub_rn(s, bv);
    e = __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv));
    return s;
}

// Float-float addition (h, l) += (bh, bl): the unevaluated sum h + l carries
// about 48 significant bits, and the error of one addition is a few units of
// 2^-48 of |h| + |bh|.  The result does not depend on the operand order.
__device__ __forceinline__ void lse_ff_add(float &h, float &l, float bh, float bl)
{
    float e;
    const float s = lse_two_sum(h, bh, e);
    e = __fadd_rn(e, __fadd_rn(l, bl));
    h = __fadd_rn(s, e);                        // |s| >= |e|: Fast2Sum
    l = __fsub_rn(e, __fsub_rn(h, s));
}

// Reduces NV per-thread compensated sums (value s[k] - c[k], lse_kahan_add)
// and two counts over the CTA in float-float arithmetic: warp shuffles in a
// fixed pattern, then warps in index order; FP64 only for the final values.
// out[k], *count0 and *count1 are valid in thread 0 after return.  NV <= 32.
template <int NV, int MAXW = 32>
__device__ __forceinline__ void lse_cta_reduce_ff(const float (&s)[NV], const float (&c)[NV],
                                                  long long n0, long long n1,
                                                  double (&out)[NV], long long *count0,
                                                  long long *count1)
{
    __shared__ float s_h[MAXW][NV], s_l[MAXW][NV];
    __shared__ long long s_n[MAXW][2];
    __shared__ double s_out[NV];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    float h[NV], l[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) h[k] = lse_two_sum(s[k], -c[k], l[k]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const float bh = __shfl_xor_sync(0xffffffffu, h[k], o);
            const float bl = __shfl_xor_sync(0xffffffffu, l[k], o);
            lse_ff_add(h[k], l[k], bh, bl);
        }
    }
    n0 = warp_sum_ll(n0);
    n1 = warp_sum_ll(n1);
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            s_h[warp][k] = h[k];
            s_l[warp][k] = l[k];
        }
        s_n[warp][0] = n0;
        s_n[warp][1] = n1;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        const int k = threadIdx.x;
        float th = 0.0f, tl = 0.0f;
        for (int w = 0; w < nwarps; ++w) lse_ff_add(th, tl, s_h[w][k], s_l[w][k]);
        s_out[k] = (double)th + (double)tl;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t0 = 0, t1 = 0;
        for (int w = 0; w < nwarps; ++w) {
            t0 += s_n[w][0];
            t1 += s_n[w][1];
        }
        *count0 = t0;
        *count1 = t1;
#pragma unroll
        for (int k = 0; k < NV; ++k) out[k] = s_out[k];
    }
    __syncthreads();
}

// Reduces `acc` over the CTA (blockDim.x a multiple of 32 and at least 64,
// at most 32 MAXW) into `out` (visible to thread 0 after return).  `nb`
// bands are summed.  MAXW sizes the static shared arrays: a kernel of few
// warps passes its own count and keeps that shared memory for its tiles.
// PAR: the per-warp results meet in one thread per value instead of thread 0.
template <int MAXW = 32, bool PAR = false>
__device__ __forceinline__ void lse_cta_reduce(const LseAcc &acc, int nb,
                                               LseAcc *out)
{
    __shared__ double s_d[MAXW][2 * LSE_MAXB];
    __shared__ long long s_l[MAXW][2];
    __shared__ float s_f[MAXW][2];
    __shared__ unsigned int s_u[MAXW];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
#pragma unroll
    for (int b = 0; b < LSE_MAXB; ++b) {
        if (b < nb) {
            double p = warp_sum_d(acc.sp[b]);
            double m = warp_sum_d(acc.sm[b]);
            if (lane == 0) {
                s_d[warp][b] = p;
                s_d[warp][LSE_MAXB + b] = m;
            }
        }
    }
    long long np = warp_sum_ll(acc.n_plus);
    long long fl = warp_sum_ll(acc.flips);
    float fx = acc.fmax, fn = acc.fmin;
    unsigned int bits = acc.bits;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        fx = fmaxf(fx, __shfl_xor_sync(0xffffffffu, fx, o));
        fn = fminf(fn, __shfl_xor_sync(0xffffffffu, fn, o));
        bits |= __shfl_xor_sync(0xffffffffu, bits, o);
    }
    if (lane == 0) {
        s_l[warp][0] = np;
        s_l[warp][1] = fl;
        s_f[warp][0] = fx;
        s_f[warp][1] = fn;
        s_u[warp] = bits;
    }
    __syncthreads();
    if constexpr (PAR) {
        // across the warps in index order, one thread per value (FP64 adds
        // have a latency of ~64 cycles on this part): for many bands at
        // the end of a one-wave pass.  The step kernels keep the one-thread
        // form, which measured faster there.
        __shared__ double s_sum[2 * LSE_MAXB];
        __shared__ long long s_cnt[2];
        const int k = threadIdx.x;
        if (k < 2 * nb) {
            const int col = k < nb ? k : LSE_MAXB + (k - nb);
            double v = 0.0;
            for (int w = 0; w < nwarps; ++w) v += s_d[w][col];
            s_sum[k] = v;
        } else if (k >= 32 && k < 34) {
            long long v = 0;
            for (int w = 0; w < nwarps; ++w) v += s_l[w][k - 32];
            s_cnt[k - 32] = v;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            out->clear();
            for (int b = 0; b < nb; ++b) {
                out->sp[b] = s_sum[b];
                out->sm[b] = s_sum[nb + b];
            }
            out->n_plus = s_cnt[0];
            out->flips = s_cnt[1];
            for (int w = 0; w < nwarps; ++w) {
                out->fmax = fmaxf(out->fmax, s_f[w][0]);
                out->fmin = fminf(out->fmin, s_f[w][1]);
                out->bits |= s_u[w];
            }
        }
    } else {
        if (threadIdx.x == 0) {
            // warps in index order, in registers (not through `out`, a
            // generic pointer the compiler must reload and store every step)
            double sp[LSE_MAXB], sm[LSE_MAXB];
#pragma unroll
            for (int b = 0; b < LSE_MAXB; ++b) sp[b] = sm[b] = 0.0;
            long long np = 0, fl = 0;
            float fx = -INFINITY, fn = INFINITY;
            unsigned int bits = 0;
            for (int w = 0; w < nwarps; ++w) {
#pragma unroll
                for (int b = 0; b < LSE_MAXB; ++b) {
                    if (b < nb) {
                        sp[b] += s_d[w][b];
                        sm[b] += s_d[w][LSE_MAXB + b];
                    }
                }
                np += s_l[w][0];
                fl += s_l[w][1];
                fx = fmaxf(fx, s_f[w][0]);
                fn = fminf(fn, s_f[w][1]);
                bits |= s_u[w];
            }
            out->clear();
#pragma unroll
            for (int b = 0; b < LSE_MAXB; ++b) {
                if (b < nb) {
                    out->sp[b] = sp[b];
                    out->sm[b] = sm[b];
                }
            }
            out->n_plus = np;
            out->flips = fl;
            out->fmax = fx;
            out->fmin = fn;
            out->bits = bits;
        }
    }
    __syncthreads();
}

__device__ __forceinline__ void lse_store_partial(const LseAcc &r, int nb,
                                                  LsePartial *p)
{
    for (int b = 0; b < LSE_MAXB; ++b) {
        p->sp[b] = b < nb ? r.sp[b] : 0.0;
        p->sm[b] = b < nb ? r.sm[b] : 0.0;
    }
    p->n_plus = r.n_plus;
    p->flips = r.flips;
    p->fmax = r.fmax;
    p->fmin = r.fmin;
    p->bits = r.bits;
}

// Writes the partial of CTA `cta` of the `ncta` CTAs reducing into `st` and
// returns true in the one that finished last.  The CTA-wide result `r` is
// only meaningful in thread 0.
__device__ __forceinline__ bool lse_publish_and_ticket_at(const LseAcc &r, int nb,
                                                          LsePartial *partials,
                                                          LseDevState *st, int cta, int ncta)
{
    __shared__ int s_last;
    if (threadIdx.x == 0) {
        lse_store_partial(r, nb, partials + cta);
        __threadfence();
        unsigned int t = atomicAdd(&st->ticket, 1u);
        s_last = (t == (unsigned int)ncta - 1);
    }
    __syncthreads();
    bool last = s_last != 0;
    if (last) __threadfence();
    return last;
}

// The same for a grid that reduces into one state record.
__device__ __forceinline__ bool lse_publish_and_ticket(const LseAcc &r, int nb,
                                                       LsePartial *partials,
                                                       LseDevState *st)
{
    return lse_publish_and_ticket_at(r, nb, partials, st, blockIdx.x, gridDim.x);
}

// In the last CTA: sums all partials in CTA order into `total` (thread 0).
template <int MAXW = 32, bool PAR = false>
__device__ __forceinline__ void lse_sum_partials(const LsePartial *partials,
                                                 int nparts, int nb,
                                                 LseAcc *total)
{
    LseAcc a;
    a.clear();
    if constexpr (PAR) {
        // every field of a partial loaded at once into register sums (band
        // loop unrolled; pass a constant nb), so the L2 latency is paid once
        // per partial rather than once per field
        double sp[LSE_MAXB], sm[LSE_MAXB];
#pragma unroll
        for (int b = 0; b < LSE_MAXB; ++b) sp[b] = sm[b] = 0.0;
        long long np = 0, fl = 0;
        float fx = -INFINITY, fn = INFINITY;
        unsigned int bits = 0;
        for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
            const LsePartial *p = partials + i;
#pragma unroll
            for (int b = 0; b < LSE_MAXB; ++b) {
                if (b < nb) {
                    sp[b] += __ldcg(&p->sp[b]);
                    sm[b] += __ldcg(&p->sm[b]);
                }
            }
            np += __ldcg(&p->n_plus);
            fl += __ldcg(&p->flips);
            fx = fmaxf(fx, __ldcg(&p->fmax));
            fn = fminf(fn, __ldcg(&p->fmin));
            bits |= __ldcg(&p->bits);
        }
#pragma unroll
        for (int b = 0; b < LSE_MAXB; ++b) {
            a.sp[b] = sp[b];
            a.sm[b] = sm[b];
        }
        a.n_plus = np;
        a.flips = fl;
        a.fmax = fx;
        a.fmin = fn;
        a.bits = bits;
    } else {
        for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
            const LsePartial *p = partials + i;
            for (int b = 0; b < nb; ++b) {
                a.sp[b] += __ldcg(&p->sp[b]);
                a.sm[b] += __ldcg(&p->sm[b]);
            }
            a.n_plus += __ldcg(&p->n_plus);
            a.flips += __ldcg(&p->flips);
            a.fmax = fmaxf(a.fmax, __ldcg(&p->fmax));
            a.fmin = fminf(a.fmin, __ldcg(&p->fmin));
            a.bits |= __ldcg(&p->bits);
        }
    }
    lse_cta_reduce<MAXW, PAR>(a, nb, total);
}

// Exact sums for the tile form.  A lane's sums over one tile are FP32
// values x with |x| <= 32 max|I| (at most 28 pixels); round(x 2^k) is taken
// from the bits of x with integer operations only and added up as 64-bit
// integers.  Integer addition is associative, so the totals do not depend on
// which CTA took which tile nor on the order of the additions, and the
// statistics are the same bits however the tiles are scheduled.  k is chosen
// per call (lse_fix_scale) so that every total fits: the rounding is 2^-k,
// about 2^-35 of max|I| at 2^26 pixels.
__device__ __forceinline__ long long lse_fix(float x, int k)
{
    const unsigned int u = __float_as_uint(x);
    const int e = (int)((u >> 23) & 255u);
    if (e == 0 || e == 255) return 0;           // zero / subnormal (< one unit); never inf
    const long long m = (long long)((u & 0x7FFFFFu) | 0x800000u);
    const int sh = e - 150 + k;                 // |x| 2^k = m 2^sh
    long long r;
    if (sh >= 0) r = m << sh;
    else if (sh >= -24) r = (m + (1ll << (-sh - 1))) >> (-sh);
    else r = 0;
    return (u >> 31) ? -r : r;
}

// The exponent k of lse_fix for N pixels of magnitude at most `maxabs`:
// sums of N values below 2^62 once scaled, and a lane's partial (at most 32
// values) too.
__host__ __device__ inline int lse_fix_scale(double maxabs, long long n)
{
    if (!(maxabs > 0.0) || !isfinite(maxabs)) return 30;
    int e;
    const double f = frexp((double)(n > 32 ? n : 32) * maxabs, &e);   // f in [0.5, 1)
    const int ceil_log2 = f == 0.5 ? e - 1 : e;
    int k = 61 - ceil_log2;
    return k < -120 ? -120 : (k > 120 ? 120 : k);
}

// The totals of a tile-form step from the fixed-point sums (slot of the
// state record): sum I over v >= 0 and over v < 0, the count and the sign
// changes.
__device__ __forceinline__ void lse_fix_totals(long long sw, long long sa, long long np,
                                               long long fl, int k, LseAcc &t)
{
    t.clear();
    t.sp[0] = ldexp((double)(sa + sw), -(k + 1));
    t.sm[0] = ldexp((double)(sa - sw), -(k + 1));
    t.n_plus = np;
    t.flips = fl;
}

// Sums NV 64-bit integers over the CTA (warp shuffles, then the warps in
// index order); the totals are valid in thread 0.
template <int NV, int MAXW>
__device__ __forceinline__ void lse_cta_sum_i64(long long (&v)[NV])
{
    __shared__ long long s_v[MAXW][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = warp_sum_ll(v[k]);
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) s_v[warp][k] = v[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            long long t = 0;
            for (int w = 0; w < MAXW; ++w) t += s_v[w][k];
            v[k] = t;
        }
    }
    __syncthreads();
}

// Means of one band over the two sides (Eq. 15) and the factors of the data
// term D = alpha (I - mid), alpha = 2 (c+ - c-), mid = (c+ + c-) / 2
// (Eq. 17's numerator).  Explicit round-to-nearest operations: every kernel
// that makes these coefficients (the last CTA of a step, every CTA of the
// persistent evolution, the band statistics pass) gets the same bits.
__device__ __forceinline__ void lse_band_coeffs(double sp, double sm, long long np, long long nm,
                                                double &cp, double &cm, double &al, double &md)
{
    cp = np > 0 ? __ddiv_rn(sp, (double)np) : 0.0;
    cm = nm > 0 ? __ddiv_rn(sm, (double)nm) : 0.0;
    al = __dmul_rn(2.0, __dsub_rn(cp, cm));
    md = __dmul_rn(0.5, __dadd_rn(cp, cm));
}

// One band: the normaliser M = |c+ - c-| max(|2 Imax - s|, |2 Imin - s|),
// s = c+ + c-, and the step coefficient dt alpha / (2 M).  Returns false
// when M is not positive (zero force).
__device__ __forceinline__ bool lse_norm_one_band(double cp, double cm, double al, double imin,
                                                  double imax, float dt, double &norm, float &a0)
{
    const double s = __dadd_rn(cp, cm);
    const double M = __dmul_rn(fabs(__dsub_rn(cp, cm)),
                               fmax(fabs(__dsub_rn(__dmul_rn(2.0, imax), s)),
                                    fabs(__dsub_rn(__dmul_rn(2.0, imin), s))));
    if (!(M > 0.0)) return false;
    norm = M;
    a0 = __double2float_rn(__ddiv_rn(__dmul_rn((double)dt, al), __dmul_rn(2.0, M)));
    return true;
}

// Region statistics of the current LSF -> c+/c- and the coefficients of the
// next step (Eqs. 15 and 17).  For one band the normaliser has the closed
// form M = |c+ - c-| max(|2 Imax - c+ - c-|, |2 Imin - c+ - c-|) (|2I - s|
// is convex in I, so its maximum over the image sits at Imin or Imax); for
// several bands M comes from the normaliser pass.  Thread 0 only.
__device__ __forceinline__ void lse_region_coeffs_v(LseDevState *st, const LseAcc &t, int B,
                                                    float dt, long long N, double imin,
                                                    double imax)
{
    // writes the state record only: a read back of a field just stored (or
    // any dependent read of the record) is a memory round trip at the end of
    // a launch, on one thread, with every other SM idle
    const long long np = t.n_plus;
    const long long nm = N - np;
    double contrast = 0.0, scale = 0.0, cp0 = 0.0, cm0 = 0.0, al0 = 0.0;
    for (int b = 0; b < B; ++b) {
        double cp, cm, al, md;
        lse_band_coeffs(t.sp[b], t.sm[b], np, nm, cp, cm, al, md);
        st->run_sp[b] = t.sp[b];
        st->run_sm[b] = t.sm[b];
        st->c_plus[b] = cp;
        st->c_minus[b] = cm;
        st->alpha[b] = al;
        st->mid[b] = md;
        st->af[b] = __double2float_rn(al);
        st->m[b] = __double2float_rn(md);
        contrast = fmax(contrast, fabs(cp - cm));
        scale = fmax(scale, fabs(cp) + fabs(cm));
        if (b == 0) {
            cp0 = cp;
            cm0 = cm;
            al0 = al;
        }
    }
    st->area_plus = np;
    int zero = (np == 0 || nm == 0 || contrast <= LSE_CONTRAST_TOL * scale);
    double norm = 0.0;
    float a0 = 0.0f;
    if (!zero && B == 1 && !lse_norm_one_band(cp0, cm0, al0, imin, imax, dt, norm, a0)) {
        zero = 1;
        norm = 0.0;
    }
    st->norm = norm;
    if (zero) {
        for (int b = 0; b < LSE_MAXB; ++b) st->a[b] = 0.0f;
    } else if (B == 1) {
        st->a[0] = a0;
    }
    st->zero_force = zero;
}

__device__ __forceinline__ void lse_region_coeffs(LseDevState *st,
                                                  const LseAcc &t, int B,
                                                  float dt)
{
    const long long N = st->npix;
    const double imin = st->imin, imax = st->imax;
    lse_region_coeffs_v(st, t, B, dt, N, imin, imax);
}

// The state fields a step's finalisation reads, loaded together (one
// latency) by thread 0 before the CTA's reduction; none of them changes
// during the step.
struct LseStatePre {
    double norm, imin, imax;
    long long npix;
    int zero_force;
};

__device__ __forceinline__ LseStatePre lse_state_pre(const LseDevState *st)
{
    LseStatePre p;
    p.norm = st->norm;
    p.imin = st->imin;
    p.imax = st->imax;
    p.npix = st->npix;
    p.zero_force = st->zero_force;
    return p;
}

// End of one executed step (thread 0 of the last CTA): record the step,
// then compute the statistics of the new LSF and the next step's
// coefficients.  `t` holds the grid-wide sums over the new LSF.
__device__ __forceinline__ void lse_step_finalize(const StepArgs &a, const LseAcc &t,
                                                  const LseStatePre &pre)
{
    LseDevState *st = a.st;
    unsigned int bits = t.bits;
    st->last_flips = t.flips;
    st->iterations_run = a.iter + 1;
    st->last_buf = a.out_buf;
    if (a.term == LSE_TERM_REGION && a.mb_split) {
        // vector image on the tile form: the next statistics pass makes the
        // coefficients of the next step
        if (pre.zero_force) bits |= LSE_SBIT_DEGENERATE;
        st->norm_used = pre.zero_force ? 0.0 : pre.norm;
        st->area_plus = t.n_plus;
    } else if (a.term == LSE_TERM_REGION) {
        if (pre.zero_force) bits |= LSE_SBIT_DEGENERATE;
        st->norm_used = pre.zero_force ? 0.0 : pre.norm;
        lse_region_coeffs_v(st, t, a.B, a.dt, pre.npix, pre.imin, pre.imax);
    } else {
        st->area_plus = t.n_plus;
    }
    if (bits) atomicOr(&st->status_bits, bits);
    if (a.early_thresh > 0.0 && (double)t.flips < a.early_thresh) st->done = 1;
    __threadfence();
    st->ticket = 0;
}

__device__ __forceinline__ void lse_step_finalize(const StepArgs &a, const LseAcc &t)
{
    lse_step_finalize(a, t, lse_state_pre(a.st));
}
