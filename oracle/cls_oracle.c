/*
 * cls_oracle.c -- plain, slow FP64 CPU oracle for Chord Length Sampling (CLS).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this library.  It shares
 * no code with the CUDA path (paper_1708_00765_gb300/csrc); the two agree
 * because both follow the same published definitions:
 *
 *   - CLS "Algorithm A" (paper Sec. 4): per flight draw the collision distance
 *     l_c ~ Exp(Sigma_m) and the interface distance l_i ~ Exp(mean Lambda_m),
 *     compute the boundary distance l_b, take the minimum, move, then either
 *     leak, collide (scatter with probability c_m, else absorb) or switch the
 *     material label.  All distances are redrawn after every event.
 *   - 3D source and isotropic scattering (paper Sec. 4.3): incident cosine law
 *     mu' = sqrt(xi), phi' uniform; scatter mu = 2 xi - 1, phi = 2 pi xi',
 *     omega = (sqrt(1-mu^2) cos phi, sqrt(1-mu^2) sin phi, mu).
 *   - Box of side L, leakage on the faces normal to x, specular reflection on
 *     the lateral faces (paper Sec. 2).
 *   - Initial material label from p_i = Lambda_i / (Lambda_0 + Lambda_1)
 *     (paper Sec. 2).
 *   - Track-length estimator of the scalar flux on a uniform x mesh, integrated
 *     over y and z, plus reflection / transmission counts (paper Sec. 2, 3.3).
 *   - Rod (d = 1): directions +-1, interface distance along the rod; isotropic
 *     scattering picks +1 or -1 with probability 1/2 each.
 *   - Suite II source (paper Sec. 2, 4.1, 4.3): position uniform in the
 *     box (x; box also y, z), direction isotropic (rod: +-1 with probability
 *     1/2; slab: mu = 2 xi - 1; box: mu = 2 xi - 1, phi = 2 pi xi', omega =
 *     (sqrt(1-mu^2) cos phi, sqrt(1-mu^2) sin phi, mu)), then the label.
 *   - Extruded 2D (d = 2, paper Sec. 4.2): the box's x and y faces only (the
 *     geometry is invariant along z); the 3D direction omega of the box, with
 *     mu = omega_z the cosine to the extrusion axis; interface distance
 *     d_i = -Lambda/sqrt(1 - mu^2) ln(1 - xi), the in-plane chord projected on
 *     the flight.  Sources draw no z (suite I: y, mu', phi'; suite II: x, y,
 *     mu, phi).
 *   - Box projected on x (d = 13): the box's x-marginal.  Specular lateral
 *     faces keep omega_x, and CLS chords are drawn along the flight, so the
 *     tallies have the law of a walk in mu = omega_x alone: incident
 *     mu = sqrt(xi), volume source mu = 2 xi - 1, scattering mu = 2 xi - 1 (the
 *     x cosine of an isotropic direction), chords not projected, x faces only.
 *   - Slab (d = 11, the paper's d = 1, Sec. 4.1): direction cosine mu with
 *     respect to x; incident mu = sqrt(xi); interface distance projected,
 *     d_i = -(Lambda/|mu|) ln(1 - xi); scattering mu = 2 xi - 1; x faces only.
 *   - Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel
 *     random numbers: as easy as 1, 2, 3", SC'11), counter
 *     (j >> 1, h_lo, h_hi, case), key (seed_lo, seed_hi); even draw j uses
 *     output words (0,1), odd j words (2,3); u = (((w_hi << 32) | w_lo) >> 11)
 *     * 2^-53.  Each draw recomputes the block from scratch: slow and plain.
 *
 * Readings where the paper is silent (tie rules, draw order, clamping) are the
 * ones listed with the design notes: boundary wins ties, then collision; an x
 * face wins over a lateral face; the collision draw is consumed even when
 * Sigma_m = 0; the scattering-decision draw is consumed for every collision.
 *
 * Flux tallies are summed per (batch, bin) with Neumaier compensation in
 * history order; batch b holds histories first + b*batch_len ...
 *
 * Build: cc -std=c11 -O2 -ffp-contract=off -fPIC -shared (no FMA contraction).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

typedef struct {
    double sigma[2];  /* total cross sections Sigma_0, Sigma_1            */
    double lambda[2]; /* mean chord lengths Lambda_0, Lambda_1            */
    double c[2];      /* scattering probability c_i = Sigma_s,i / Sigma_i */
    double L;         /* rod length / box side                           */
    int32_t d;        /* 1 rod, 2 extruded 2D, 3 box, 11 slab, 13 box (x only) */
    int32_t nbins;    /* uniform x bins for the flux tally               */
    int32_t source;   /* 0 = incident flux on x = 0 (suite I),           */
                      /* 1 = uniform isotropic volume source (suite II)   */
    int32_t pad;
} orc_case_t;

typedef struct {
    uint64_t n_histories, nR, nT, nA, n_coll, n_int, n_refl, n_events, max_events, n_capped;
    double sum_t;    /* sum over histories of the total track length      */
    double sum_t2;   /* sum over histories of its square                  */
    double track[2]; /* total track length spent in material 0 / 1        */
} orc_counts_t;

/* event codes used in traces */
enum { EV_LEAK_X0 = 0, EV_LEAK_XL = 1, EV_REFLECT = 2, EV_SCATTER = 3, EV_ABSORB = 4, EV_INTERFACE = 5, EV_CAPPED = 6 };

/* ---------------------------------------------------------------- Philox */

/* Philox4x32 with 10 rounds, as defined by Salmon et al. (SC'11): each round
 * multiplies words 0 and 2 by the two round constants, takes high and low
 * halves, and mixes with words 1, 3 and the round key; the key is bumped by
 * the Weyl constants between rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

typedef struct {
    uint32_t key[2];
    uint32_t h_lo, h_hi, case_id;
    uint64_t j; /* per-history draw index */
} orc_stream_t;

/* draw number j of the history: uniform in [0, 1) with 53 random bits */
double orc_uniform(uint64_t seed, uint32_t case_id, uint64_t h, uint64_t j)
{
    uint32_t ctr[4] = {(uint32_t)(j >> 1), (uint32_t)h, (uint32_t)(h >> 32), case_id};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    uint32_t hi = (j & 1) ? w[2] : w[0];
    uint32_t lo = (j & 1) ? w[3] : w[1];
    uint64_t bits = ((uint64_t)hi << 32) | (uint64_t)lo;
    return (double)(bits >> 11) * 0x1p-53;
}

static double next_u(orc_stream_t *s)
{
    uint64_t seed = ((uint64_t)s->key[1] << 32) | s->key[0];
    uint64_t h = ((uint64_t)s->h_hi << 32) | s->h_lo;
    double u = orc_uniform(seed, s->case_id, h, s->j);
    s->j++;
    return u;
}

/* ------------------------------------------------------ compensated sums */

typedef struct { double s, c; } nsum_t;

static void nsum_add(nsum_t *a, double v)
{
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v))
        a->c += (a->s - t) + v;
    else
        a->c += (v - t) + a->s;
    a->s = t;
}

static double nsum_get(const nsum_t *a) { return a->s + a->c; }

/* ------------------------------------------------------------- tallies */

typedef struct {
    const orc_case_t *cs;
    nsum_t *bins;       /* [nbins] of the current batch */
    nsum_t track[2];
    double t_hist;      /* total track length of the current history */
} orc_tally_t;

/* bin edge e_k = k L / nbins */
static double edge(const orc_case_t *cs, int k) { return ((double)k * cs->L) / (double)cs->nbins; }

/* Track-length estimator: a flight of length l in material m from x0 to x1
 * with direction cosine wx deposits in bin k the path length inside the slab
 * e_k <= x < e_{k+1}: overlap(x-extent) / |wx|.  A flight that lies inside one
 * bin deposits its length l itself (the same path length, free of the
 * cancellation overlap/|wx| suffers for grazing flights, |wx| -> 0).  The
 * x-extent is clipped to the box [0, L].  A flight with wx == 0 puts its whole
 * length into the bin containing x0. */
static void tally_flight(orc_tally_t *t, double x0, double x1, double wx, double l, int m)
{
    const orc_case_t *cs = t->cs;
    t->t_hist += l;
    nsum_add(&t->track[m], l);
    if (l <= 0.0)
        return;
    if (wx == 0.0) {
        int k = (int)floor(x0 * (double)cs->nbins / cs->L);
        if (k < 0) k = 0;
        if (k > cs->nbins - 1) k = cs->nbins - 1;
        nsum_add(&t->bins[k], l);
        return;
    }
    double lo = x0 < x1 ? x0 : x1;
    double hi = x0 < x1 ? x1 : x0;
    if (lo < 0.0) lo = 0.0;
    if (hi > cs->L) hi = cs->L;
    double aw = fabs(wx);
    /* only bins whose edges can overlap [lo, hi] are visited; the overlap
     * formula itself is the definition */
    int k0 = (int)floor(lo * (double)cs->nbins / cs->L) - 1;
    int k1 = (int)floor(hi * (double)cs->nbins / cs->L) + 1;
    if (k0 < 0) k0 = 0;
    if (k1 > cs->nbins - 1) k1 = cs->nbins - 1;
    for (int k = k0; k <= k1; k++) {
        double a = lo > edge(cs, k) ? lo : edge(cs, k);
        double b = hi < edge(cs, k + 1) ? hi : edge(cs, k + 1);
        if (b > a)
            nsum_add(&t->bins[k], (a == lo && b == hi) ? l : (b - a) / aw);
    }
}

/* ------------------------------------------------------------- traces */

typedef struct {
    double *rows;
    int cap, n;
} orc_trace_t;

static void trace_event(orc_trace_t *tr, int ev, const orc_stream_t *s, const double r[3],
                        const double w[3], int m, double l)
{
    if (!tr || tr->n >= tr->cap)
        return;
    double *row = tr->rows + 10 * tr->n;
    row[0] = ev;
    row[1] = (double)s->j;
    row[2] = r[0]; row[3] = r[1]; row[4] = r[2];
    row[5] = w[0]; row[6] = w[1]; row[7] = w[2];
    row[8] = m;
    row[9] = l;
    tr->n++;
}

/* ------------------------------------------------------------ history */

/* Outcome of one history: 0 = reflected, 1 = transmitted, 2 = absorbed,
 * 3 = event cap reached. */
static int run_history(const orc_case_t *cs, uint32_t case_id, uint64_t seed, uint64_t h,
                       uint64_t max_events, orc_tally_t *tal, orc_counts_t *cnt, orc_trace_t *tr)
{
    orc_stream_t s;
    s.key[0] = (uint32_t)seed;
    s.key[1] = (uint32_t)(seed >> 32);
    s.h_lo = (uint32_t)h;
    s.h_hi = (uint32_t)(h >> 32);
    s.case_id = case_id;
    s.j = 0;

    const double L = cs->L;
    const double p0 = cs->lambda[0] / (cs->lambda[0] + cs->lambda[1]);
    double r[3] = {0.0, 0.0, 0.0};
    double w[3] = {1.0, 0.0, 0.0};

    /* source: position and direction first, then the material label */
    if (cs->source == 1) {
        r[0] = L * next_u(&s);
        if (cs->d == 3 || cs->d == 2) {
            r[1] = L * next_u(&s);
            if (cs->d == 3)
                r[2] = L * next_u(&s);
            double mu = 2.0 * next_u(&s) - 1.0;
            double ph = (2.0 * ORC_PI) * next_u(&s);
            double st = sqrt(1.0 - mu * mu);
            w[0] = st * cos(ph);
            w[1] = st * sin(ph);
            w[2] = mu;
        } else if (cs->d == 11 || cs->d == 13) {
            w[0] = 2.0 * next_u(&s) - 1.0;
        } else {
            w[0] = (next_u(&s) < 0.5) ? 1.0 : -1.0;
        }
    } else if (cs->d == 11 || cs->d == 13) {
        w[0] = sqrt(next_u(&s)); /* cosine law mu = sqrt(xi) */
    } else if (cs->d == 3 || cs->d == 2) {
        r[1] = L * next_u(&s);
        if (cs->d == 3)
            r[2] = L * next_u(&s);
        double mu = sqrt(next_u(&s));
        double ph = (2.0 * ORC_PI) * next_u(&s);
        double st = sqrt(1.0 - mu * mu);
        w[0] = mu;
        w[1] = st * cos(ph);
        w[2] = st * sin(ph);
    }
    int m = (next_u(&s) < p0) ? 0 : 1;

    uint64_t events = 0;
    int outcome = -1;
    while (outcome < 0) {
        if (events == max_events) {
            outcome = 3;
            trace_event(tr, EV_CAPPED, &s, r, w, m, 0.0);
            break;
        }
        events++;

        /* collision and interface distances, in this order */
        double u_c = next_u(&s);
        double l_c = (cs->sigma[m] > 0.0) ? -log(1.0 - u_c) / cs->sigma[m] : INFINITY;
        double u_i = next_u(&s);
        double l_i = -cs->lambda[m] * log(1.0 - u_i);
        if (cs->d == 11)
            l_i = l_i / fabs(w[0]); /* projection of the chord on x */
        else if (cs->d == 2)
            l_i = l_i / sqrt(1.0 - w[2] * w[2]); /* in-plane chord along the flight */

        /* boundary distance: x faces, then (box) the lateral faces */
        double l_b = INFINITY;
        int face = -1; /* 0: x = 0, 1: x = L, 2: lateral */
        if (w[0] > 0.0) { l_b = (L - r[0]) / w[0]; face = 1; }
        else if (w[0] < 0.0) { l_b = (0.0 - r[0]) / w[0]; face = 0; }
        if (l_b < 0.0) l_b = 0.0;
        double l_lat[3] = {INFINITY, INFINITY, INFINITY};
        if (cs->d == 3 || cs->d == 2) {
            int na = (cs->d == 3) ? 3 : 2; /* extruded: y faces only */
            for (int a = 1; a < na; a++) {
                if (w[a] > 0.0) l_lat[a] = (L - r[a]) / w[a];
                else if (w[a] < 0.0) l_lat[a] = (0.0 - r[a]) / w[a];
                if (l_lat[a] < 0.0) l_lat[a] = 0.0;
                if (l_lat[a] < l_b) { l_b = l_lat[a]; face = 2; }
            }
        }

        if (l_b <= l_c && l_b <= l_i) {
            /* boundary */
            double x0 = r[0];
            if (face == 0 || face == 1) {
                double xf = (face == 0) ? 0.0 : L;
                tally_flight(tal, x0, xf, w[0], l_b, m);
                r[0] = xf;
                r[1] += l_b * w[1];
                if (cs->d == 3)
                    r[2] += l_b * w[2];
                if (face == 0) { cnt->nR++; outcome = 0; trace_event(tr, EV_LEAK_X0, &s, r, w, m, l_b); }
                else { cnt->nT++; outcome = 1; trace_event(tr, EV_LEAK_XL, &s, r, w, m, l_b); }
            } else {
                double x1 = r[0] + l_b * w[0];
                tally_flight(tal, x0, x1, w[0], l_b, m);
                r[0] = x1;
                for (int a = 1; a < 3; a++) {
                    if (l_lat[a] == l_b) {
                        r[a] = (w[a] > 0.0) ? L : 0.0; /* snap onto the face */
                        w[a] = -w[a];                  /* specular reflection */
                    } else if (a == 1 || cs->d == 3) {
                        r[a] += l_b * w[a];
                    }
                }
                cnt->n_refl++;
                trace_event(tr, EV_REFLECT, &s, r, w, m, l_b);
            }
        } else {
            double l = (l_c <= l_i) ? l_c : l_i;
            double x0 = r[0];
            double x1 = r[0] + l * w[0];
            tally_flight(tal, x0, x1, w[0], l, m);
            r[0] = x1;
            r[1] += l * w[1];
            if (cs->d == 3)
                r[2] += l * w[2];
            if (l_c <= l_i) {
                /* collision: scatter with probability c_m, else absorb */
                cnt->n_coll++;
                if (next_u(&s) < cs->c[m]) {
                    if (cs->d == 1) {
                        w[0] = (next_u(&s) < 0.5) ? 1.0 : -1.0;
                    } else if (cs->d == 11 || cs->d == 13) {
                        w[0] = 2.0 * next_u(&s) - 1.0;
                    } else {
                        double mu = 2.0 * next_u(&s) - 1.0;
                        double ph = (2.0 * ORC_PI) * next_u(&s);
                        double st = sqrt(1.0 - mu * mu);
                        w[0] = st * cos(ph);
                        w[1] = st * sin(ph);
                        w[2] = mu;
                    }
                    trace_event(tr, EV_SCATTER, &s, r, w, m, l);
                } else {
                    cnt->nA++;
                    outcome = 2;
                    trace_event(tr, EV_ABSORB, &s, r, w, m, l);
                }
            } else {
                /* interface: switch the material label */
                m = 1 - m;
                cnt->n_int++;
                trace_event(tr, EV_INTERFACE, &s, r, w, m, l);
            }
        }
    }
    if (outcome == 3)
        cnt->n_capped++;
    cnt->n_events += events;
    if (events > cnt->max_events)
        cnt->max_events = events;
    return outcome;
}

static int check_case(const orc_case_t *cs)
{
    if (!cs) return -1;
    if (cs->d != 1 && cs->d != 2 && cs->d != 3 && cs->d != 11 && cs->d != 13) return -1;
    if (cs->nbins < 1) return -1;
    if (cs->source != 0 && cs->source != 1) return -1;
    if (!(cs->L > 0.0)) return -1;
    for (int i = 0; i < 2; i++) {
        if (!(cs->sigma[i] >= 0.0) || !isfinite(cs->sigma[i])) return -1;
        if (!(cs->lambda[i] > 0.0) || !isfinite(cs->lambda[i])) return -1;
        if (!(cs->c[i] >= 0.0 && cs->c[i] <= 1.0)) return -1;
    }
    return 0;
}

/* Run histories first .. first+n-1 of one case.
 *   flux   : [nbatch][nbins] raw track-length sums (caller-owned, overwritten)
 *   history h goes to batch (h - first) / batch_len
 * Returns 0, or -1 on invalid input. */
int orc_run(const orc_case_t *cs, uint32_t case_id, uint64_t seed, uint64_t first, uint64_t n,
            uint64_t max_events, uint64_t batch_len, uint32_t nbatch, orc_counts_t *out, double *flux)
{
    if (check_case(cs) || !out || !flux || batch_len == 0 || nbatch == 0)
        return -1;
    if ((n + batch_len - 1) / batch_len > nbatch)
        return -1;
    size_t nb = (size_t)cs->nbins;
    nsum_t *bins = calloc(nb * nbatch, sizeof(nsum_t));
    if (!bins)
        return -1;
    memset(out, 0, sizeof(*out));
    orc_tally_t tal;
    memset(&tal, 0, sizeof(tal));
    tal.cs = cs;
    nsum_t st = {0, 0}, st2 = {0, 0};
    for (uint64_t i = 0; i < n; i++) {
        tal.bins = bins + nb * (size_t)(i / batch_len);
        tal.t_hist = 0.0;
        run_history(cs, case_id, seed, first + i, max_events, &tal, out, NULL);
        nsum_add(&st, tal.t_hist);
        nsum_add(&st2, tal.t_hist * tal.t_hist);
    }
    out->n_histories = n;
    out->sum_t = nsum_get(&st);
    out->sum_t2 = nsum_get(&st2);
    out->track[0] = nsum_get(&tal.track[0]);
    out->track[1] = nsum_get(&tal.track[1]);
    for (size_t k = 0; k < nb * nbatch; k++)
        flux[k] = nsum_get(&bins[k]);
    free(bins);
    return 0;
}

/* Outcome of each of histories first .. first+n-1 of one case, one byte per
 * history (0 reflected, 1 transmitted, 2 absorbed, 3 event cap; paper Sec. 2
 * observables R, T, A).  Tallies are computed and discarded.
 * Returns 0, or -1 on invalid input. */
int orc_outcomes(const orc_case_t *cs, uint32_t case_id, uint64_t seed, uint64_t first, uint64_t n,
                 uint64_t max_events, uint8_t *codes)
{
    if (check_case(cs) || !codes)
        return -1;
    size_t nb = (size_t)cs->nbins;
    nsum_t *bins = calloc(nb, sizeof(nsum_t));
    if (!bins)
        return -1;
    orc_counts_t cnt;
    memset(&cnt, 0, sizeof(cnt));
    orc_tally_t tal;
    memset(&tal, 0, sizeof(tal));
    tal.cs = cs;
    tal.bins = bins;
    for (uint64_t i = 0; i < n; i++) {
        tal.t_hist = 0.0;
        codes[i] = (uint8_t)run_history(cs, case_id, seed, first + i, max_events, &tal, &cnt, NULL);
    }
    free(bins);
    return 0;
}

/* Event-by-event trace of history h: rows of 10 doubles
 * (event, draw index after the event, x, y, z, wx, wy, wz, material, flight length).
 * Returns the number of rows written (at most cap), or -1 on invalid input. */
int orc_trace(const orc_case_t *cs, uint32_t case_id, uint64_t seed, uint64_t h, uint64_t max_events,
              double *rows, int cap, orc_counts_t *out)
{
    if (check_case(cs) || !rows || cap < 0 || !out)
        return -1;
    size_t nb = (size_t)cs->nbins;
    nsum_t *bins = calloc(nb, sizeof(nsum_t));
    if (!bins)
        return -1;
    memset(out, 0, sizeof(*out));
    orc_tally_t tal;
    memset(&tal, 0, sizeof(tal));
    tal.cs = cs;
    tal.bins = bins;
    orc_trace_t tr = {rows, cap, 0};
    run_history(cs, case_id, seed, h, max_events, &tal, out, &tr);
    out->n_histories = 1;
    out->sum_t = tal.t_hist;
    out->sum_t2 = tal.t_hist * tal.t_hist;
    out->track[0] = nsum_get(&tal.track[0]);
    out->track[1] = nsum_get(&tal.track[1]);
    free(bins);
    return tr.n;
}
