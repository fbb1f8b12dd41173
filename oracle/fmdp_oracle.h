/*
 * FastMDP first-come-first-served planning: plain FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark load this library. The GPU scheduler never calls it and
 * shares no code, header, table or constant generator with it.
 *
 * Paper: Bertram, Zambreno, Wei, "Scalable FastMDP for Pre-departure Airspace
 * Reservation and Strategic De-conflict" (arXiv 2008.03518).
 *   value of a state ........ Alg. 1 (FastMDP), Alg. 4-8 (reward and value kernels)
 *   peaks ................... Sec. III peak tuple {r, gamma, p, R}; Table 3
 *   forward projection ...... Alg. 1, Alg. 3
 *   action selection ........ Alg. 1, Alg. 9
 *   terminal / collision .... Sec. IV "Determine terminal state"; Sec. V
 *   FCFS admission .......... Sec. I and Sec. V (accept only conflict-free plans)
 */
#ifndef FMDP_ORACLE_H
#define FMDP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_ACTIONS 64
#define ORC_MAX_WELLS 16

enum { ORC_ADMITTED = 0, ORC_REJ_CONFLICT = 1, ORC_REJ_TERRAIN = 2, ORC_REJ_HORIZON = 3,
       ORC_REJ_NO_ACTION = 4 };

typedef struct {
    double x0, y0, z0, x1, y1, z1;   /* airspace box (m) */
    double dt;                        /* step length (s) */
    double gamma;                     /* MDP discount = decay of the goal peak */
    double goal_reward;               /* |r| of the goal peak */
    double deck_value;                /* hard-deck constant: penalty = deck_value - clearance */
    double clearance;                 /* terrain clearance below which the penalty applies */
    double sep_h, sep_v;              /* separation minima (m) */
    int32_t combine;                  /* 0: max over negative peaks (paper); 1: sum */
    int32_t n_actions;
    double dpsi_deg[ORC_MAX_ACTIONS]; /* heading change per step, multiple of 15 deg */
    double climb[ORC_MAX_ACTIONS];    /* climb rate (m/s) */
    int32_t n_wells;                  /* risk wells per known plan */
    double w_tau[ORC_MAX_WELLS];      /* well centre = p + tau * v (s) */
    double w_radius[ORC_MAX_WELLS];
    double w_mag[ORC_MAX_WELLS];      /* |r| */
    double w_gamma[ORC_MAX_WELLS];
    int32_t hm_nx, hm_ny;             /* heightmap nodes (0 = no terrain) */
    const float* heightmap;           /* [hm_ny][hm_nx], copied at create */
    int32_t n_static;
    const double* static_wells;       /* [n_static][6] x,y,z,R,|r|,gamma; copied at create */
    int32_t lookahead_W;              /* projected sub-steps per action (0 or 1: one) */
} orc_params;

typedef struct {
    double ox, oy, oz, gx, gy, gz, speed;
    int64_t depart;
    int32_t horizon;
} orc_request;

typedef struct {
    int32_t verdict;          /* ORC_* */
    int32_t n_points;         /* trajectory points incl. the origin */
    int32_t captured;
    int32_t near_ties;        /* steps whose top-2 gap was below the near-tie bar */
    int32_t followed_ties;    /* near-ties where a supplied action differed from the own argmax */
    int32_t mismatch_step;    /* first step where a supplied action was NOT a near-tie (-1 none) */
    int32_t first_conflict;   /* trajectory index of the first separation loss (-1 none) */
    int32_t first_terrain;    /* trajectory index of the first point below terrain (-1 none) */
    double min_sep_h, min_sep_v;
    int64_t plan_id;          /* admitted id, -1 otherwise */
    int64_t well_tests;       /* (action, plan, well) distance evaluations performed */
} orc_result;

typedef struct orc_t orc_t;

orc_t* orc_create(const orc_params* p);
void orc_destroy(orc_t* o);
int64_t orc_add_plan(orc_t* o, int64_t t0, const float* xyz, int32_t n);
int32_t orc_n_plans(const orc_t* o);
/* Threads that value a step's actions (OpenMP build; the results do not depend on it).
 * Returns the number in effect (1 without OpenMP). Process-wide. */
int32_t orc_set_threads(int32_t n);

/* Unit heading vectors for the 24 headings psi0 + k*15 deg, psi0 = bearing origin->goal. */
void orc_heading_table(double ox, double oy, double gx, double gy, double* C, double* S);
/* Bilinear terrain height (0 without a heightmap). */
double orc_terrain(const orc_t* o, double x, double y);

/* Q for every action from state (s, heading index h) at time step t; successors are
 * scored against known plans at t+1. Outputs per action (arrays of n_actions):
 * Q (-inf if invalid), goal term g, negative-peak aggregate P, hard-deck V, valid, and
 * successor states nxt[3*a]. Returns the number of (action, plan, well) tests. */
int64_t orc_q_values(const orc_t* o, const double* s, int32_t h, int64_t t, double speed,
                     const double* goal, const double* C, const double* S,
                     double* Q, double* g, double* P, double* V, int32_t* valid, double* nxt);

/* Greedy FastMDP rollout of one request. If follow != NULL (length n_follow) the rollout
 * takes follow[k] at step k whenever it is a near-tie with the own argmax (lock-step
 * parity); a non-tie disagreement is recorded in mismatch_step and the own argmax is used.
 * Buffers (capacity cap points / steps; may be NULL): xyz fp32 [cap][3], states fp64
 * [cap][3], headings [cap], actions [cap], q_trace [cap][n_actions], scale_trace
 * [cap][n_actions] (per-action term scale max(g, P+V)), tie_flags [cap]. */
int32_t orc_rollout(const orc_t* o, const orc_request* r, const int32_t* follow, int32_t n_follow,
                    int32_t cap, float* xyz, double* states, int32_t* headings, int32_t* actions,
                    double* q_trace, double* scale_trace, int32_t* tie_flags, orc_result* res);

/* Separation and terrain check of a trajectory (fp32 points from slice t0) against every
 * known plan. Fills first_conflict, first_terrain, min_sep_h, min_sep_v. Returns the number
 * of conflicting (point, plan) pairs. */
int64_t orc_sep_check(const orc_t* o, int64_t t0, const float* xyz, int32_t n, orc_result* res);

/* Co-simulation of n requests on one clock, each seeing the others' Table 3 wells at their
 * current position and velocity (no admission). follow: optional [n][cap] actions (-1: none)
 * taken at near-ties as in orc_rollout. Buffers [n][cap][3] / [n][cap] / [n][cap][A] (may be
 * NULL); res[i].verdict is -1 for a captured request, else HORIZON or NO_ACTION. */
int32_t orc_cosim(const orc_t* o, const orc_request* reqs, int32_t n, const int32_t* follow, int32_t cap,
                  float* xyz, int32_t* actions, double* q_trace, double* scale_trace, orc_result* res);

/* FCFS: rollout, separation check, and admission of a conflict-free trajectory. */
int32_t orc_schedule(orc_t* o, const orc_request* r, int32_t cap, float* xyz, int32_t* actions,
                     orc_result* res);

#ifdef __cplusplus
}
#endif
#endif
