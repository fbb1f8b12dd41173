/*
 * FastMDP first-come-first-served planning: plain FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark load this library; the GPU scheduler never calls it and the
 * two share no code. Compiled with -ffp-contract=off so that every floating-point
 * expression below is evaluated exactly as written (IEEE round-to-nearest, no fused
 * multiply-add), on any host.
 *
 * What it computes, in the paper's order (Bertram, Zambreno, Wei, arXiv 2008.03518):
 *  1. Peaks (Sec. III, peak tuple {r, gamma, p, R}; Table 3): a goal peak of magnitude
 *     goal_reward and decay gamma with infinite radius, and for every known plan j that
 *     is present at the successor time t+1, one risk well per row of the well table,
 *     centred at p_j + tau * v_j (Table 3 "p + v t"), with v_j the plan's own velocity
 *     (p_j(t+2) - p_j(t+1)) / dt, or 0 when the plan has ended at t+2. Static wells
 *     (terrain / restricted volumes, Table 3 terrain row) are fixed peaks.
 *  2. Forward projection (Alg. 1, Alg. 3): each action turns the heading by a multiple
 *     of 15 degrees, then moves speed*dt horizontally and climb*dt vertically.
 *  3. Value of each successor (Alg. 1; Alg. 4-8): V = |r_g| gamma^d_goal
 *        - AGG over negative peaks of [d < R] |r| gamma_r^d - V_deck,
 *     AGG = max (Alg. 5-8 keep the atomic maximum per class and Alg. 8 takes the max
 *     of the classes) or, as an option, the sum. V_deck is the hard-deck penalty of
 *     Alg. 1 evaluated at the successor against terrain clearance.
 *  4. Action selection (Alg. 1, Alg. 9): argmax over valid actions, lowest index on
 *     ties; the state advances to the chosen successor.
 *  4'. Lookahead window W (Sec. IV "Forward project", Alg. 9): each action is held for W
 *     sub-steps of dt, giving W projected states x_1 .. x_W (x_j = x_(j-1) plus the same
 *     per-step move); x_j is valued against the peaks at time t + j, and the action's
 *     value is the largest of the values of its projected states inside the box. The
 *     action is valid when x_1 is inside the box, and the state advances to x_1 of the
 *     chosen action (one step of dt). W = 1 is items 2-4 above.
 *  5. Terminal test (Sec. IV "Determine terminal state", Sec. V): the goal is captured
 *     when within one step (speed*dt) of it; the request fails if the horizon runs out
 *     or no action is valid.
 *  6. FCFS admission (Sec. I, Sec. V): the finished trajectory is accepted only if no
 *     sample is within the separation minima of any known plan at the same time step
 *     and no sample is below terrain; an accepted trajectory becomes a known plan.
 *
 * Readings where the paper is silent or inconsistent (heading table, capture radius,
 * window W = 1 at dt = 1 s, velocity from the stored plan, strict inequalities) are
 * the ones stated in the repository's design notes.
 */
#include "fmdp_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define TIE_REL 1e-4

typedef struct {
    int64_t t0;
    int32_t n;
    float* xyz;
    int64_t id;
} orc_plan;

struct orc_t {
    orc_params p;
    float* hm;
    double* statics;
    int32_t dh[ORC_MAX_ACTIONS]; /* heading change in 15-degree units */
    orc_plan* plans;
    int32_t n_plans, cap_plans;
    int64_t next_id;
};

orc_t* orc_create(const orc_params* p) {
    if (!p || p->n_actions < 1 || p->n_actions > ORC_MAX_ACTIONS || p->n_wells < 0 ||
        p->n_wells > ORC_MAX_WELLS || p->dt <= 0.0)
        return NULL;
    orc_t* o = (orc_t*)calloc(1, sizeof(orc_t));
    o->p = *p;
    for (int a = 0; a < p->n_actions; ++a) {
        double q = p->dpsi_deg[a] / 15.0;
        long k = lround(q);
        if (fabs(q - (double)k) > 1e-9) { free(o); return NULL; }
        o->dh[a] = (int32_t)k;
    }
    if (p->hm_nx >= 2 && p->hm_ny >= 2 && p->heightmap) {
        size_t n = (size_t)p->hm_nx * (size_t)p->hm_ny;
        o->hm = (float*)malloc(n * sizeof(float));
        memcpy(o->hm, p->heightmap, n * sizeof(float));
    } else {
        o->p.hm_nx = o->p.hm_ny = 0;
    }
    if (p->n_static > 0 && p->static_wells) {
        o->statics = (double*)malloc((size_t)p->n_static * 6 * sizeof(double));
        memcpy(o->statics, p->static_wells, (size_t)p->n_static * 6 * sizeof(double));
    } else {
        o->p.n_static = 0;
    }
    o->p.heightmap = o->hm;
    o->p.static_wells = o->statics;
    o->next_id = 1;
    return o;
}

void orc_destroy(orc_t* o) {
    if (!o) return;
    for (int32_t i = 0; i < o->n_plans; ++i) free(o->plans[i].xyz);
    free(o->plans);
    free(o->hm);
    free(o->statics);
    free(o);
}

int64_t orc_add_plan(orc_t* o, int64_t t0, const float* xyz, int32_t n) {
    if (!o || n < 1 || !xyz) return -1;
    if (o->n_plans == o->cap_plans) {
        o->cap_plans = o->cap_plans ? 2 * o->cap_plans : 256;
        o->plans = (orc_plan*)realloc(o->plans, (size_t)o->cap_plans * sizeof(orc_plan));
    }
    orc_plan* pl = &o->plans[o->n_plans++];
    pl->t0 = t0;
    pl->n = n;
    pl->xyz = (float*)malloc((size_t)n * 3 * sizeof(float));
    memcpy(pl->xyz, xyz, (size_t)n * 3 * sizeof(float));
    pl->id = o->next_id++;
    return pl->id;
}

int32_t orc_n_plans(const orc_t* o) { return o ? o->n_plans : 0; }

/* Unit vectors of the 24 headings psi0 + k*15 deg. psi0 is the bearing from origin to
 * goal; cos/sin of multiples of 15 deg come from their surd forms and are rotated onto
 * psi0 with plain products, so the table is reproducible bit for bit. */
void orc_heading_table(double ox, double oy, double gx, double gy, double* C, double* S) {
    double r2 = sqrt(2.0), r3 = sqrt(3.0), r6 = sqrt(6.0);
    double c15 = (r6 + r2) / 4.0, s15 = (r6 - r2) / 4.0;
    double qc[6] = {1.0, c15, r3 / 2.0, r2 / 2.0, 0.5, s15};
    double qs[6] = {0.0, s15, 0.5, r2 / 2.0, r3 / 2.0, c15};
    double dx = gx - ox, dy = gy - oy;
    double L = sqrt(dx * dx + dy * dy);
    double c0 = 1.0, s0 = 0.0;
    if (L > 0.0) { c0 = dx / L; s0 = dy / L; }
    for (int k = 0; k < 24; ++k) {
        int quad = k / 6, m = k % 6;
        double ck, sk; /* cos, sin of k*15 deg */
        if (quad == 0)      { ck = qc[m];  sk = qs[m]; }
        else if (quad == 1) { ck = -qs[m]; sk = qc[m]; }
        else if (quad == 2) { ck = -qc[m]; sk = -qs[m]; }
        else                { ck = qs[m];  sk = -qc[m]; }
        C[k] = c0 * ck - s0 * sk;
        S[k] = s0 * ck + c0 * sk;
    }
}

/* Bilinear interpolation of the heightmap, nodes spanning the airspace box. */
double orc_terrain(const orc_t* o, double x, double y) {
    const orc_params* p = &o->p;
    if (p->hm_nx < 2) return 0.0;
    int nx = p->hm_nx, ny = p->hm_ny;
    double fx = (x - p->x0) / (p->x1 - p->x0) * (double)(nx - 1);
    double fy = (y - p->y0) / (p->y1 - p->y0) * (double)(ny - 1);
    double flx = floor(fx), fly = floor(fy);
    int ix = (int)flx, iy = (int)fly;
    if (flx < 0.0) ix = 0;
    if (fly < 0.0) iy = 0;
    if (ix > nx - 2) ix = nx - 2;
    if (iy > ny - 2) iy = ny - 2;
    double ax = fx - (double)ix, ay = fy - (double)iy;
    double h00 = o->hm[(size_t)iy * nx + ix], h10 = o->hm[(size_t)iy * nx + ix + 1];
    double h01 = o->hm[(size_t)(iy + 1) * nx + ix], h11 = o->hm[(size_t)(iy + 1) * nx + ix + 1];
    return (1.0 - ay) * ((1.0 - ax) * h00 + ax * h10) + ay * ((1.0 - ax) * h01 + ax * h11);
}

/* Position of plan pl at time step t, if it has a sample there. */
static int plan_at(const orc_plan* pl, int64_t t, double* q) {
    int64_t k = t - pl->t0;
    if (k < 0 || k >= pl->n) return 0;
    q[0] = (double)pl->xyz[3 * k];
    q[1] = (double)pl->xyz[3 * k + 1];
    q[2] = (double)pl->xyz[3 * k + 2];
    return 1;
}

/* One negative peak: [d < R] |r| gamma^d (Alg. 5-7), folded into the running aggregate. */
static double fold_peak(const orc_params* p, double agg, double d, double R, double mag, double gam) {
    if (!(d < R)) return agg;
    double val = mag * pow(gam, d);
    if (p->combine) return agg + val;
    return val > agg ? val : agg;
}

/* The three terms of the value of a state (x, y, z) scored at time step tn: the goal
 * peak (Alg. 4), the aggregate of negative peaks of the known plans present at tn and of
 * the static wells (Alg. 5-7), and the hard-deck penalty (Alg. 1). */
/* Extra negative peaks of one step: the wells of the other aircraft of a co-simulated batch
 * (centres xc[3 * i], well row xk[i] of the well table). */
typedef struct {
    const double* xc;
    const int32_t* xk;
    int32_t n;
} orc_extra;

static void state_terms(const orc_t* o, double x, double y, double z, int64_t tn, const double* goal,
                        const orc_extra* ex_peaks, double* g_out, double* P_out, double* V_out, int64_t* tests) {
    const orc_params* p = &o->p;
    {
        /* positive peak: the goal (Alg. 4), |r| gamma^d with infinite radius */
        double ex = goal[0] - x, ey = goal[1] - y, ez = goal[2] - z;
        double dg = sqrt(ex * ex + ey * ey + ez * ez);
        *g_out = p->goal_reward * pow(p->gamma, dg);

        /* negative peaks of known plans (Alg. 7, Table 3 wells) */
        double agg = 0.0;
        for (int32_t j = 0; j < o->n_plans; ++j) {
            const orc_plan* pl = &o->plans[j];
            double p1[3], p2[3], v[3] = {0.0, 0.0, 0.0};
            if (!plan_at(pl, tn, p1)) continue;
            if (plan_at(pl, tn + 1, p2)) {
                v[0] = (p2[0] - p1[0]) / p->dt;
                v[1] = (p2[1] - p1[1]) / p->dt;
                v[2] = (p2[2] - p1[2]) / p->dt;
            }
            for (int k = 0; k < p->n_wells; ++k) {
                double cx = p1[0] + p->w_tau[k] * v[0];
                double cy = p1[1] + p->w_tau[k] * v[1];
                double cz = p1[2] + p->w_tau[k] * v[2];
                double dx = x - cx, dy = y - cy, dz = z - cz;
                double d = sqrt(dx * dx + dy * dy + dz * dz);
                ++*tests;
                agg = fold_peak(p, agg, d, p->w_radius[k], p->w_mag[k], p->w_gamma[k]);
            }
        }
        /* the other aircraft of a co-simulated batch (Alg. 1 "build neg rewards", Build
         * Peaks kernel: Table 3 wells at their current position and velocity) */
        if (ex_peaks)
            for (int32_t i = 0; i < ex_peaks->n; ++i) {
                const double* c = ex_peaks->xc + 3 * i;
                int k = ex_peaks->xk[i];
                double dx = x - c[0], dy = y - c[1], dz = z - c[2];
                double d = sqrt(dx * dx + dy * dy + dz * dz);
                ++*tests;
                agg = fold_peak(p, agg, d, p->w_radius[k], p->w_mag[k], p->w_gamma[k]);
            }
        /* static negative peaks: terrain / restricted volumes (Alg. 6) */
        for (int32_t w = 0; w < p->n_static; ++w) {
            const double* sw = &o->statics[6 * w];
            double dx = x - sw[0], dy = y - sw[1], dz = z - sw[2];
            double d = sqrt(dx * dx + dy * dy + dz * dz);
            agg = fold_peak(p, agg, d, sw[3], sw[4], sw[5]);
        }
        *P_out = agg;

        /* hard deck (Alg. 1) as terrain clearance at the state */
        double vd = 0.0;
        if (p->hm_nx >= 2) {
            double c = z - orc_terrain(o, x, y);
            if (c < p->clearance) vd = p->deck_value - c;
        }
        *V_out = vd;
    }
}

/* threads over which a step's actions are valued (1: the plain sequential loop) */
static int g_threads = 1;

int32_t orc_set_threads(int32_t n) {
#ifdef _OPENMP
    g_threads = n > 1 ? n : 1;
#else
    g_threads = 1;
#endif
    return g_threads;
}

static int in_box(const orc_params* p, double x, double y, double z) {
    return x >= p->x0 && x <= p->x1 && y >= p->y0 && y <= p->y1 && z >= p->z0 && z <= p->z1;
}

static int64_t q_values_x(const orc_t* o, const double* s, int32_t h, int64_t t, double speed,
                          const double* goal, const double* C, const double* S, const orc_extra* ex_peaks,
                          double* Q, double* g, double* P, double* V, int32_t* valid, double* nxt) {
    const orc_params* p = &o->p;
    double step = speed * p->dt;
    int W = p->lookahead_W > 1 ? p->lookahead_W : 1;
    int64_t tests = 0;
    /* the actions' values are independent of one another: with OpenMP (orc_set_threads) the
     * actions are shared out over threads; every value is computed exactly as written */
#ifdef _OPENMP
#pragma omp parallel for schedule(static) reduction(+ : tests) if (g_threads > 1) num_threads(g_threads)
#endif
    for (int a = 0; a < p->n_actions; ++a) {
        /* forward projection (Alg. 3): turn, then move */
        int hn = ((h + o->dh[a]) % 24 + 24) % 24;
        double x = s[0] + step * C[hn];
        double y = s[1] + step * S[hn];
        double z = s[2] + p->climb[a] * p->dt;
        nxt[3 * a] = x; nxt[3 * a + 1] = y; nxt[3 * a + 2] = z;
        int ok = in_box(p, x, y, z);
        valid[a] = ok;
        /* value of x_1, then of x_2 .. x_W (the action held), keeping the largest */
        state_terms(o, x, y, z, t + 1, goal, ex_peaks, &g[a], &P[a], &V[a], &tests);
        double best = g[a] - P[a] - V[a];
        for (int j = 2; j <= W; ++j) {
            x = x + step * C[hn];
            y = y + step * S[hn];
            z = z + p->climb[a] * p->dt;
            if (!in_box(p, x, y, z)) continue;
            double gj, Pj, Vj;
            state_terms(o, x, y, z, t + j, goal, ex_peaks, &gj, &Pj, &Vj, &tests);
            double vj = gj - Pj - Vj;
            if (vj > best) {
                best = vj;
                g[a] = gj;
                P[a] = Pj;
                V[a] = Vj;
            }
        }
        Q[a] = ok ? best : -INFINITY;
    }
    return tests;
}

int64_t orc_q_values(const orc_t* o, const double* s, int32_t h, int64_t t, double speed,
                     const double* goal, const double* C, const double* S,
                     double* Q, double* g, double* P, double* V, int32_t* valid, double* nxt) {
    return q_values_x(o, s, h, t, speed, goal, C, S, NULL, Q, g, P, V, valid, nxt);
}

static double term_scale(double g, double P, double V) {
    double n = P + V;
    return g > n ? g : n;
}

static int near_tie(double q1, double q2, double s1, double s2) {
    double m = fabs(q1);
    if (fabs(q2) > m) m = fabs(q2);
    if (s1 > m) m = s1;
    if (s2 > m) m = s2;
    return (q1 - q2) < TIE_REL * m;
}

int32_t orc_rollout(const orc_t* o, const orc_request* r, const int32_t* follow, int32_t n_follow,
                    int32_t cap, float* xyz, double* states, int32_t* headings, int32_t* actions,
                    double* q_trace, double* scale_trace, int32_t* tie_flags, orc_result* res) {
    const orc_params* p = &o->p;
    int A = p->n_actions;
    memset(res, 0, sizeof(*res));
    res->verdict = -1;
    res->mismatch_step = -1;
    res->first_conflict = -1;
    res->first_terrain = -1;
    res->plan_id = -1;
    if (r->horizon < 0 || cap < r->horizon + 1 || r->speed <= 0.0) return -1;

    double C[24], S[24];
    orc_heading_table(r->ox, r->oy, r->gx, r->gy, C, S);
    double goal[3] = {r->gx, r->gy, r->gz};
    double s[3] = {r->ox, r->oy, r->oz};
    int32_t h = 0;
    int64_t t = r->depart;
    double step = r->speed * p->dt;
    double cap2 = step * step;

    double Q[ORC_MAX_ACTIONS], g[ORC_MAX_ACTIONS], P[ORC_MAX_ACTIONS], V[ORC_MAX_ACTIONS];
    double nxt[3 * ORC_MAX_ACTIONS];
    int32_t valid[ORC_MAX_ACTIONS];

    int32_t n = 0;
#define PUT_POINT()                                                              \
    do {                                                                         \
        if (xyz) { xyz[3 * n] = (float)s[0]; xyz[3 * n + 1] = (float)s[1];       \
                   xyz[3 * n + 2] = (float)s[2]; }                               \
        if (states) { states[3 * n] = s[0]; states[3 * n + 1] = s[1];            \
                      states[3 * n + 2] = s[2]; }                                \
        if (headings) headings[n] = h;                                           \
        ++n;                                                                     \
    } while (0)
    PUT_POINT();

    double ex = goal[0] - s[0], ey = goal[1] - s[1], ez = goal[2] - s[2];
    int captured = (ex * ex + ey * ey + ez * ez) <= cap2;
    for (int32_t k = 0; k < r->horizon && !captured; ++k) {
        res->well_tests += orc_q_values(o, s, h, t, r->speed, goal, C, S, Q, g, P, V, valid, nxt);
        int a1 = -1, a2 = -1;
        for (int a = 0; a < A; ++a)
            if (valid[a] && (a1 < 0 || Q[a] > Q[a1])) a1 = a;
        if (a1 < 0) { res->verdict = ORC_REJ_NO_ACTION; break; }
        for (int a = 0; a < A; ++a)
            if (a != a1 && valid[a] && (a2 < 0 || Q[a] > Q[a2])) a2 = a;
        double s1 = term_scale(g[a1], P[a1], V[a1]);
        int tie = a2 >= 0 && near_tie(Q[a1], Q[a2], s1, term_scale(g[a2], P[a2], V[a2]));
        if (tie) res->near_ties++;
        if (tie_flags) tie_flags[k] = tie;
        if (q_trace) for (int a = 0; a < A; ++a) q_trace[(size_t)k * A + a] = Q[a];
        if (scale_trace)
            for (int a = 0; a < A; ++a) scale_trace[(size_t)k * A + a] = term_scale(g[a], P[a], V[a]);

        int chosen = a1;
        if (follow && k < n_follow && follow[k] != a1) {
            int fa = follow[k];
            if (fa >= 0 && fa < A && valid[fa] &&
                near_tie(Q[a1], Q[fa], s1, term_scale(g[fa], P[fa], V[fa]))) {
                chosen = fa;
                res->followed_ties++;
            } else if (res->mismatch_step < 0) {
                res->mismatch_step = k;
            }
        }
        if (actions) actions[k] = chosen;
        h = ((h + o->dh[chosen]) % 24 + 24) % 24;
        s[0] = nxt[3 * chosen]; s[1] = nxt[3 * chosen + 1]; s[2] = nxt[3 * chosen + 2];
        ++t;
        PUT_POINT();
        ex = goal[0] - s[0]; ey = goal[1] - s[1]; ez = goal[2] - s[2];
        captured = (ex * ex + ey * ey + ez * ez) <= cap2;
    }
#undef PUT_POINT
    res->n_points = n;
    res->captured = captured;
    if (res->verdict < 0 && !captured) res->verdict = ORC_REJ_HORIZON;
    return 0;
}

int64_t orc_sep_check(const orc_t* o, int64_t t0, const float* xyz, int32_t n, orc_result* res) {
    const orc_params* p = &o->p;
    double hh = p->sep_h * p->sep_h;
    int64_t conflicts = 0;
    res->first_conflict = -1;
    res->first_terrain = -1;
    res->min_sep_h = INFINITY;
    res->min_sep_v = INFINITY;
    for (int32_t k = 0; k < n; ++k) {
        double a[3] = {(double)xyz[3 * k], (double)xyz[3 * k + 1], (double)xyz[3 * k + 2]};
        if (p->hm_nx >= 2 && res->first_terrain < 0 && a[2] < orc_terrain(o, a[0], a[1]))
            res->first_terrain = k;
        for (int32_t j = 0; j < o->n_plans; ++j) {
            double q[3];
            if (!plan_at(&o->plans[j], t0 + k, q)) continue;
            double dx = a[0] - q[0], dy = a[1] - q[1], dz = fabs(a[2] - q[2]);
            double h2 = dx * dx + dy * dy;
            if (dz < p->sep_v) {
                double hd = sqrt(h2);
                if (hd < res->min_sep_h) res->min_sep_h = hd;
            }
            if (h2 < hh) {
                if (dz < res->min_sep_v) res->min_sep_v = dz;
                if (dz < p->sep_v) {
                    ++conflicts;
                    if (res->first_conflict < 0) res->first_conflict = k;
                }
            }
        }
    }
    return conflicts;
}

int32_t orc_schedule(orc_t* o, const orc_request* r, int32_t cap, float* xyz, int32_t* actions,
                     orc_result* res) {
    if (orc_rollout(o, r, NULL, 0, cap, xyz, NULL, NULL, actions, NULL, NULL, NULL, res) != 0)
        return -1;
    orc_result chk;
    orc_sep_check(o, r->depart, xyz, res->n_points, &chk);
    res->first_conflict = chk.first_conflict;
    res->first_terrain = chk.first_terrain;
    res->min_sep_h = chk.min_sep_h;
    res->min_sep_v = chk.min_sep_v;
    if (res->verdict < 0) {
        if (chk.first_conflict >= 0) res->verdict = ORC_REJ_CONFLICT;
        else if (chk.first_terrain >= 0) res->verdict = ORC_REJ_TERRAIN;
        else res->verdict = ORC_ADMITTED;
    }
    if (res->verdict == ORC_ADMITTED) res->plan_id = orc_add_plan(o, r->depart, xyz, res->n_points);
    return 0;
}

/* Co-simulation of a batch (Alg. 1 "DistributedUam"; Sec. V, batches whose aircraft see
 * each other). All aircraft step on one clock: at step t every aircraft in flight (departed,
 * not finished) values its actions against the known plans, the static peaks and the
 * Table 3 wells of every other aircraft in flight, centred at that aircraft's position at t
 * plus tau times its velocity (its last move over dt; zero before its first move). Then all
 * of them take their chosen actions together. Admission is left to the caller. */
int32_t orc_cosim(const orc_t* o, const orc_request* reqs, int32_t n, const int32_t* follow, int32_t cap,
                  float* xyz, int32_t* actions, double* q_trace, double* scale_trace, orc_result* res) {
    const orc_params* p = &o->p;
    const int A = p->n_actions, K = p->n_wells;
    if (n <= 0) return 0;
    for (int32_t i = 0; i < n; ++i)
        if (reqs[i].horizon < 0 || cap < reqs[i].horizon + 1 || reqs[i].speed <= 0.0) return -1;
    double* C = malloc(sizeof(double) * 24 * n);
    double* S = malloc(sizeof(double) * 24 * n);
    double* st = malloc(sizeof(double) * 3 * n);
    double* prev = malloc(sizeof(double) * 3 * n);
    int32_t* h = calloc(n, sizeof(int32_t));
    int32_t* k = calloc(n, sizeof(int32_t));
    int32_t* done = calloc(n, sizeof(int32_t));
    int32_t* choice = malloc(sizeof(int32_t) * n);
    double* nx = malloc(sizeof(double) * 3 * n);
    double* xc = malloc(sizeof(double) * 3 * (size_t)K * n);
    int32_t* xk = malloc(sizeof(int32_t) * (size_t)K * n);
    int32_t* owner = malloc(sizeof(int32_t) * (size_t)K * n);
    double* xc_i = malloc(sizeof(double) * 3 * (size_t)K * n);
    int32_t* xk_i = malloc(sizeof(int32_t) * (size_t)K * n);
    if (!C || !S || !st || !prev || !h || !k || !done || !choice || !nx || !xc || !xk || !owner || !xc_i || !xk_i) {
        free(C); free(S); free(st); free(prev); free(h); free(k); free(done); free(choice); free(nx);
        free(xc); free(xk); free(owner); free(xc_i); free(xk_i);
        return -1;
    }
    int64_t t = reqs[0].depart;
    for (int32_t i = 0; i < n; ++i) {
        const orc_request* r = &reqs[i];
        orc_heading_table(r->ox, r->oy, r->gx, r->gy, C + 24 * i, S + 24 * i);
        st[3 * i] = r->ox; st[3 * i + 1] = r->oy; st[3 * i + 2] = r->oz;
        memset(&res[i], 0, sizeof(orc_result));
        res[i].verdict = -1;
        res[i].mismatch_step = -1;
        res[i].first_conflict = -1;
        res[i].first_terrain = -1;
        res[i].plan_id = -1;
        res[i].n_points = 1;
        if (xyz) {
            xyz[(size_t)3 * cap * i] = (float)r->ox;
            xyz[(size_t)3 * cap * i + 1] = (float)r->oy;
            xyz[(size_t)3 * cap * i + 2] = (float)r->oz;
        }
        double step = r->speed * p->dt;
        double ex = r->gx - r->ox, ey = r->gy - r->oy, ez = r->gz - r->oz;
        if ((ex * ex + ey * ey + ez * ez) <= step * step) { done[i] = 1; res[i].captured = 1; }
        else if (r->horizon <= 0) { done[i] = 1; res[i].verdict = ORC_REJ_HORIZON; }
        if (r->depart < t) t = r->depart;
    }
    double Q[ORC_MAX_ACTIONS], g[ORC_MAX_ACTIONS], P[ORC_MAX_ACTIONS], V[ORC_MAX_ACTIONS];
    double nxt[3 * ORC_MAX_ACTIONS];
    int32_t valid[ORC_MAX_ACTIONS];
    for (;;) {
        int any = 0;
        for (int32_t i = 0; i < n; ++i) any |= !done[i];
        if (!any) break;
        /* peaks of the aircraft in flight at t */
        int32_t np = 0;
        for (int32_t m = 0; m < n; ++m) {
            if (done[m] || reqs[m].depart > t) continue;
            double v[3] = {0.0, 0.0, 0.0};
            if (k[m] > 0)
                for (int c = 0; c < 3; ++c) v[c] = (st[3 * m + c] - prev[3 * m + c]) / p->dt;
            for (int w = 0; w < K; ++w) {
                for (int c = 0; c < 3; ++c) xc[3 * np + c] = st[3 * m + c] + p->w_tau[w] * v[c];
                xk[np] = w;
                owner[np] = m;
                ++np;
            }
        }
        /* every aircraft in flight chooses (against the others' peaks) */
        for (int32_t i = 0; i < n; ++i) {
            choice[i] = -1;
            if (done[i] || reqs[i].depart > t) continue;
            const orc_request* r = &reqs[i];
            orc_extra ex = {xc_i, xk_i, 0};
            for (int32_t q = 0; q < np; ++q) {
                if (owner[q] == i) continue;
                xc_i[3 * ex.n] = xc[3 * q]; xc_i[3 * ex.n + 1] = xc[3 * q + 1]; xc_i[3 * ex.n + 2] = xc[3 * q + 2];
                xk_i[ex.n] = xk[q];
                ++ex.n;
            }
            double goal[3] = {r->gx, r->gy, r->gz};
            res[i].well_tests += q_values_x(o, st + 3 * i, h[i], t, r->speed, goal, C + 24 * i, S + 24 * i, &ex, Q, g,
                                            P, V, valid, nxt);
            int a1 = -1, a2 = -1;
            for (int a = 0; a < A; ++a)
                if (valid[a] && (a1 < 0 || Q[a] > Q[a1])) a1 = a;
            const int kk = k[i];
            if (q_trace) for (int a = 0; a < A; ++a) q_trace[((size_t)i * cap + kk) * A + a] = Q[a];
            if (scale_trace)
                for (int a = 0; a < A; ++a) scale_trace[((size_t)i * cap + kk) * A + a] = term_scale(g[a], P[a], V[a]);
            if (a1 < 0) { choice[i] = -2; continue; }
            for (int a = 0; a < A; ++a)
                if (a != a1 && valid[a] && (a2 < 0 || Q[a] > Q[a2])) a2 = a;
            double s1 = term_scale(g[a1], P[a1], V[a1]);
            if (a2 >= 0 && near_tie(Q[a1], Q[a2], s1, term_scale(g[a2], P[a2], V[a2]))) res[i].near_ties++;
            int chosen = a1;
            const int32_t* fol = follow ? follow + (size_t)i * cap : NULL;
            if (fol && fol[kk] >= 0 && fol[kk] != a1) {
                int fa = fol[kk];
                if (fa < A && valid[fa] && near_tie(Q[a1], Q[fa], s1, term_scale(g[fa], P[fa], V[fa]))) {
                    chosen = fa;
                    res[i].followed_ties++;
                } else if (res[i].mismatch_step < 0) {
                    res[i].mismatch_step = kk;
                }
            }
            choice[i] = chosen;
            nx[3 * i] = nxt[3 * chosen]; nx[3 * i + 1] = nxt[3 * chosen + 1]; nx[3 * i + 2] = nxt[3 * chosen + 2];
        }
        /* all of them move together */
        for (int32_t i = 0; i < n; ++i) {
            if (choice[i] == -1) continue;
            const orc_request* r = &reqs[i];
            if (choice[i] == -2) { done[i] = 1; res[i].verdict = ORC_REJ_NO_ACTION; continue; }
            const int a = choice[i];
            if (actions) actions[(size_t)i * cap + k[i]] = a;
            for (int c = 0; c < 3; ++c) { prev[3 * i + c] = st[3 * i + c]; st[3 * i + c] = nx[3 * i + c]; }
            h[i] = ((h[i] + o->dh[a]) % 24 + 24) % 24;
            k[i] += 1;
            res[i].n_points = k[i] + 1;
            if (xyz) {
                float* pt = xyz + ((size_t)i * cap + k[i]) * 3;
                pt[0] = (float)st[3 * i]; pt[1] = (float)st[3 * i + 1]; pt[2] = (float)st[3 * i + 2];
            }
            double step = r->speed * p->dt;
            double ex = r->gx - st[3 * i], ey = r->gy - st[3 * i + 1], ez = r->gz - st[3 * i + 2];
            if ((ex * ex + ey * ey + ez * ez) <= step * step) { done[i] = 1; res[i].captured = 1; }
            else if (k[i] >= r->horizon) { done[i] = 1; res[i].verdict = ORC_REJ_HORIZON; }
        }
        ++t;
    }
    free(C); free(S); free(st); free(prev); free(h); free(k); free(done); free(choice); free(nx);
    free(xc); free(xk); free(owner); free(xc_i); free(xk_i);
    return 0;
}
