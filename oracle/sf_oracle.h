/*
 * sf_oracle.h -- plain FP64 CPU oracle of the batched multi-world vehicle step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this file: only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline leg use it.  It shares no code, header, table or constant with the
 * CUDA library; every constant below is typed here from the paper (SceneFactory,
 * arXiv 2605.08528) or from the reading stated beside it.
 *
 * The oracle is the algorithm written out in double precision, one agent and
 * one world at a time, with brute-force scans and full sorts.  Where the method
 * has a plain definition (nearest segment, k nearest points, SAT overlap) the
 * oracle is that definition; the coupled 3-D vehicle step has no closed form and
 * follows the substep order stated in sf_oracle.c.
 *
 * Layouts (row-major, one row per agent):
 *   F[A][OR_NF]  float state  (see OR_F_* indices)
 *   I[A][OR_NI]  int32 state  (see OR_I_* indices)
 *   actions[A][3] = (throttle, steer, brake), each in [-1, 1]
 *   obs[A][OR_OBS]
 */
#ifndef SF_ORACLE_H
#define SF_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* float state columns */
enum {
    OR_F_PX = 0, OR_F_PY, OR_F_PZ,           /* CoM position, world frame [m]      */
    OR_F_QW, OR_F_QX, OR_F_QY, OR_F_QZ,      /* attitude quaternion (w, x, y, z)   */
    OR_F_VX, OR_F_VY, OR_F_VZ,               /* CoM velocity [m/s]                 */
    OR_F_WX, OR_F_WY, OR_F_WZ,               /* angular velocity, world [rad/s]    */
    OR_F_S0, OR_F_S1, OR_F_S2, OR_F_S3,      /* wheel spin FL FR RL RR [rad/s]     */
    OR_F_DELTA, OR_F_DDELTA,                 /* steer angle [rad], rate [rad/s]    */
    OR_F_GX, OR_F_GY,                        /* goal [m]                           */
    OR_F_SX, OR_F_SY,                        /* episode start position [m]         */
    OR_F_MU,                                 /* friction coefficient               */
    OR_F_PEAK_DRAC,                          /* episode peak DRAC [m/s^2]          */
    OR_NF
};
/* int state columns */
enum {
    OR_I_PRECIP = 0,   /* table model: 0 dry, 1 light rain, 2 heavy rain, 3 snow;
                          ALL model: water film thickness in 0.01 mm            */
    OR_I_SURFACE,      /* table model: 0 asphalt, 1 concrete, 2 gravel;
                          ALL model: 0 AC, 1 SMA, 2 OGFC                        */
    OR_I_STEP,         /* control steps since spawn                 */
    OR_I_EPISODE,      /* episode counter of this agent slot        */
    OR_I_STATUS,       /* bit0 alive, bit1 parked                   */
    OR_I_EVENTS,       /* event bits of the last step               */
    OR_NI
};
#define OR_ALIVE  1
#define OR_PARKED 2

/* event bits */
#define OR_EV_GOAL       (1u << 0)
#define OR_EV_COLLISION  (1u << 1)
#define OR_EV_CRASH      (1u << 2)
#define OR_EV_LANE_FORB  (1u << 3)
#define OR_EV_OFFROAD    (1u << 4)
#define OR_EV_IDLE       (1u << 5)
#define OR_EV_TIMEOUT    (1u << 6)
#define OR_EV_NONFINITE  (1u << 7)
#define OR_EV_RESPAWNED  (1u << 8)

/* step flags */
#define OR_FLAG_INVINCIBLE 1
#define OR_FLAG_AUTO_RESET 2
#define OR_FLAG_BICYCLE    4   /* kinematic bicycle dynamics instead of the raycast vehicle */

#define OR_K_AGENTS 8
#define OR_L_POINTS 32
#define OR_EGO 16
#define OR_NBR_F 10
#define OR_PT_F 7
#define OR_OBS (OR_EGO + OR_K_AGENTS * OR_NBR_F + OR_L_POINTS * OR_PT_F) /* 320 */

/* Vehicle, actuation, reward and reset constants (double). */
typedef struct {
    double g, mass, half_len, half_wid, half_hgt;
    double inertia[3];            /* body-frame principal inertia (x, y, z)   */
    double hard_x, hard_y, hard_z;/* hardpoint offsets |x|, |y|, z            */
    double wheel_r, k_susp, c_susp, rest_len;
    double wheel_inertia;
    double steer_inertia, theta_max, kp, kd, tau_steer_max;
    double tau_drive, tau_brk_f, tau_brk_r;
    double lambda_yaw, lambda_lat;
    double u_z_min;               /* ray/plane grazing cut-off                 */
    double k_contact, c_contact;  /* footprint penalty contact                 */
    double damp_ramp;             /* compression over which dampers engage      */
    double wheelbase;
    /* reward / event constants (App. G) */
    double goal_radius, w_goal, w_collision, w_crash, w_lane_forb;
    double w_progress, progress_clip, w_lane, lane_sigma, lane_wh;
    double w_offroad, offroad_lat, offroad_dist, w_idle, idle_speed;
    double ttc_alpha_v, ttc_pmax_v, ttc_floor, ttc_max;
    double ttc_alpha_e, ttc_pmax_e, edge_horizon;
    double drac_thresh, w_drac, drac_gap_floor;
    double drift_max, tilt_gz;
    double seg_gap_max, scene_half, edge_half_width;
    int warmup_steps, max_steps;
    /* reset constants */
    double spawn_goal_min, spawn_goal_max, spawn_v_min, spawn_v_max;
    double spawn_spacing, park_x;
    int spawn_tries;
    double mu_table[4][3];        /* [precip][surface] */
    /* kinematic bicycle backend (Sec. 4.4 vehicle dynamics ablation) */
    double bike_theta_max;        /* steering limit, 30 degrees                                  */
    double bike_a_drive;          /* full-throttle acceleration: both front drive torques / (r m) */
    double bike_a_brake;          /* full-brake deceleration: all four brake torques / (r m)      */
    /* weather-to-friction model (Sec. 3.3, App. B): OR_WEATHER_TABLE uses mu_table;
     * OR_WEATHER_ALL the modified ALL model's static friction at 13.89 m/s */
    int weather_model;
    double all_mu[3][9];          /* mu_static at h = 0, 0.1, ..., 0.8 mm, [AC, SMA, OGFC] (App. B fig.) */
    double all_h_cut;             /* film [mm] from which the model predicts full grip loss (F5)        */
    double all_floor;             /* simulator floor of mu (App. B)                                      */
    double all_theta[3];          /* texture influence coefficient theta (App. B presets)                */
    double all_td[3];             /* texture amplitude T_d [mm] (App. B presets)                          */
    double h_norm;                /* film normaliser of the weather token [mm] (Eq. weather_obs)         */
    double stribeck_b[4];         /* b1..b4 of Eq. app_stribeck_speed                                    */
} or_params;
#define OR_WEATHER_TABLE 0
#define OR_WEATHER_ALL 1

/* Roads and agents of all worlds, as CSR (world -> polylines -> points). */
typedef struct {
    int num_worlds;
    const int32_t* agent_off;   /* [W+1] agents of world w: [agent_off[w], agent_off[w+1])   */
    const int32_t* poly_off;    /* [W+1] polylines of world w                                 */
    const int32_t* point_off;   /* [NPoly+1] points of polyline p (global point indices)      */
    const int32_t* poly_type;   /* [NPoly] Waymo type code (1,2 lane; 15,16 road edge; ...)   */
    const double* px;           /* [NPt] world-local x [m]                                    */
    const double* py;           /* [NPt] world-local y [m]                                    */
} or_scene;

/* outputs of a step / observation pass; any pointer may be NULL */
typedef struct {
    double* obs;          /* [A][OR_OBS]            */
    double* reward;       /* [A]                    */
    uint8_t* done;        /* [A]                    */
    uint32_t* events;     /* [A]                    */
    int32_t* lane_seg;    /* [A] nearest lane segment (global start-point index) or -1   */
    int32_t* knn_pts;     /* [A][OR_L_POINTS] global point indices or -1                 */
    int32_t* knn_agents;  /* [A][OR_K_AGENTS] global agent indices or -1                 */
    double* drac;         /* [A] step DRAC                                               */
} or_out;

void or_default_params(or_params* P);

/* SplitMix64 finaliser (Steele, Lea, Flood 2014), the counter-based generator of resets. */
uint64_t or_splitmix64(uint64_t x);

/* One substep of every alive agent of world w (contact forces, then each body). */
void or_substep_world(const or_params* P, const or_scene* S, int w, double* F, const int32_t* I,
                      const double* actions, double h);

/* One control step of every world: substeps, events and rewards, done agents
 * parked or respawned, then observations.  Returns the number of agents whose
 * state went non-finite. */
int or_step(const or_params* P, const or_scene* S, double* F, int32_t* I, const double* actions,
            double dt, int substeps, uint64_t seed, int flags, or_out* out);

/* Events and rewards of every alive agent, given the positions prev_xy[A][2] at
 * the start of the step and the current (end of step) state; no state change
 * except the step counter and peak DRAC.  Used for discrete parity. */
void or_events(const or_params* P, const or_scene* S, double* F, int32_t* I, const double* prev_xy,
               int flags, or_out* out);

/* Observations of every agent for the current state. */
void or_observe(const or_params* P, const or_scene* S, const double* F, const int32_t* I, or_out* out);

/* Respawn every agent with mask[a] != 0 (in agent order, world by world), then
 * observe every agent. */
void or_reset(const or_params* P, const or_scene* S, double* F, int32_t* I, const uint8_t* mask,
              uint64_t seed, or_out* out);

/* Place agent a at (x, y) with heading psi and speed v0 along the heading, at
 * the static equilibrium height, wheels rolling, goal (gx, gy). */
void or_place_agent(const or_params* P, double* F, int32_t* I, int a, double x, double y, double psi,
                    double v0, double gx, double gy, int precip, int surface);

/* --- the paper's full observation (App. D, 1,929 values per agent) --------------------
 * ego (11):    goal in the body frame / 100 (2), sin and cos of the goal bearing, goal
 *              distance / 100, body-frame velocity / 10 (2), then the weather token
 *              (precip / 3, one-hot asphalt, concrete, gravel) in place of Eq. weather_obs
 * road (350 x 5): midpoints of the world's road segments (App. C segment rule) within
 *              10 m of the CoM, in ascending segment index (polyline order), first 350:
 *              body-frame offset / 10 (2), polyline type / 20, body-frame unit direction (2)
 * vehicles (24 x 7): the 24 nearest alive other agents (ascending squared distance,
 *              ties lowest index): body-frame offset / 100 (2), length / 100, width / 100,
 *              relative heading / pi, speed / 10, swept-circle TTC / 10
 * Padding slots are zero; n_road / n_veh give the number of filled slots (a prefix). */
#define OR_FULL_EGO 11
#define OR_FULL_KR 350
#define OR_FULL_PT 5
#define OR_FULL_KV 24
#define OR_FULL_NB 7
#define OR_FULL_OBS (OR_FULL_EGO + OR_FULL_KR * OR_FULL_PT + OR_FULL_KV * OR_FULL_NB) /* 1929 */
#define OR_FULL_RADIUS 10.0

/* obs [A][OR_FULL_OBS]; n_road, n_veh [A]; road_idx [A][OR_FULL_KR] (segment start point,
 * global index) and veh_idx [A][OR_FULL_KV] (agent index), -1 padded; any may be NULL.
 * Parked / inactive agents get zeros and counts 0. */
void or_observe_full(const or_params* P, const or_scene* S, const double* F, const int32_t* I, double* obs,
                     int32_t* n_road, int32_t* n_veh, int32_t* road_idx, int32_t* veh_idx);

/* One control step of the kinematic bicycle for one agent's state row f (the
 * drop-in backend of Sec. 4.4): front-wheel steer delta = theta_bike * steer,
 * acceleration a = a_drive * throttle - a_brake * brake (both rectified), and
 * with the centre of mass midway between the axles (l_r = WB / 2) the slip angle
 * beta = atan(tan(delta) / 2); then
 *   v'   = max(0, |v| + a dt)
 *   x'   = x + v' cos(psi + beta) dt,   y' = y + v' sin(psi + beta) dt
 *   psi' = psi + (v' / l_r) sin(beta) dt
 * The row is rewritten level at the static ride height with velocity
 * v' (cos(psi' + beta), sin(psi' + beta)), yaw rate (v' / l_r) sin(beta),
 * rolling wheels v' / r_w and steer angle delta.  No suspension, contact
 * response or lateral slip. */
void or_bicycle_agent(const or_params* P, double* f, const double* act, double dt);

/* --- pieces exported for the pins ------------------------------------------------- */
/* 2-D SAT of two footprints; returns penetration depth (0 when separated), normal i->j. */
double or_sat(const or_params* P, const double ci[2], const double hi[2], const double cj[2],
              const double hj[2], double n_out[2]);
/* nearest lane segment of world w to point q: returns segment index (or -1); dist, lateral. */
int or_nearest_lane(const or_params* P, const or_scene* S, int w, const double q[2], double* dist,
                    double* lateral, double tangent[2]);
/* swept three-circle time to collision between two agents (XY), clamped to [0, ttc_max]. */
double or_ttc(const or_params* P, const double pi[2], const double hi[2], const double vi[2],
              const double pj[2], const double hj[2], const double vj[2]);
/* DRAC of j relative to i (headings hi, hj set each footprint's reach along the line of centres). */
double or_drac(const or_params* P, const double pi[2], const double hi[2], const double vi[2], const double pj[2],
               const double hj[2], const double vj[2]);
double or_lane_keep_q(const or_params* P, double lateral, double cos_dpsi);
/* circle geometry of the TTC test for a box of length L, width W, wheelbase WB. */
void or_ttc_circles(double L, double W, double WB, double* r, double* d);
/* Modified ALL model (App. B): static friction of surface s (0 AC, 1 SMA,
 * 2 OGFC) at a water film of film_cmm hundredths of a millimetre, and the
 * Stribeck speed v_s [m/s] at a film of h_m metres (Eq. app_stribeck_speed). */
double or_all_mu_static(const or_params* P, int surface, int film_cmm);
double or_stribeck_vs(const or_params* P, double h_m);
double or_penalty(double alpha, double tau, double tau_floor, double pmax);

#ifdef __cplusplus
}
#endif
#endif
