/*
 * sf_oracle.c -- plain FP64 CPU oracle of the SceneFactory vehicle step
 * (arXiv 2605.08528).  TEST INFRASTRUCTURE ONLY: only tests/, the smoke check
 * and the CPU-baseline leg of the benchmark call it; the product path never
 * does.  It shares no code with the CUDA library.
 *
 * What the paper fixes and what is a reading
 * -------------------------------------------
 * The paper simulates the vehicle as a PhysX articulation (Sec. 3.2) and gives
 * its actuation (Eq. steer_pd, App. F Tab. app_action_params), its rewards and
 * terminations (App. G Tab. app_reward_terms), its observations (App. D) and
 * its reset rule (App. J "Teleport-only reset", App. G "Termination").  It does
 * not give a tire model, contact solver or integrator.  The vehicle model here
 * is a raycast spring-damper suspension against the flat road plane z = 0
 * (roads are z-flattened, App. C), friction-capped tire impulses, and
 * semi-implicit (symplectic) Euler integration of a 6-DOF chassis, four wheel
 * spins and one steering angle over fixed substeps (120 Hz physics, 30 Hz
 * control, Sec. 4.1).  Every choice the paper leaves open is marked R<n>
 * beside the code that makes it, with its reason.
 *
 * Parity pins (tests/test_oracle_*.py): static sag m g/(4k), exact equilibrium,
 * free fall recurrence, locked-wheel stopping distance v^2/(2 mu g), the friction
 * circle invariant, kinematic yaw rate, coasting invariance, the steering
 * recurrence, SAT against polygon clipping, nearest segment and k-NN against
 * brute-force sorts, DRAC and TTC hand cases, the TTC circle geometry of App. D,
 * lane-keep score values of App. G.  The coupled 3-D step beyond these is
 * parity unpinned: no published trajectory exists, so the oracle is its own
 * authority there.
 */
#include "sf_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define INF_D 1.0e300

void or_default_params(or_params* P) {
    memset(P, 0, sizeof(*P));
    P->g = 9.81;                       /* R1: gravity, not stated in the paper                 */
    P->mass = 1500.0;                  /* sprung mass of the workload (paper's car: 1800 kg)   */
    P->half_len = 2.25;                /* 4.5 m box                                             */
    P->half_wid = 0.9;                 /* 1.8 m box                                             */
    P->half_hgt = 0.25;                /* R2: 0.5 m box height                                  */
    /* uniform box inertia m/12 (b^2 + c^2) */
    P->inertia[0] = P->mass / 12.0 * (1.8 * 1.8 + 0.5 * 0.5);
    P->inertia[1] = P->mass / 12.0 * (4.5 * 4.5 + 0.5 * 0.5);
    P->inertia[2] = P->mass / 12.0 * (4.5 * 4.5 + 1.8 * 1.8);
    P->hard_x = 1.3;                   /* half of the 2.6 m wheelbase (Sec. 3.2)                */
    P->hard_y = 0.8;                   /* R4: 1.6 m track                                       */
    P->hard_z = -0.25;                 /* hardpoints on the chassis floor                       */
    P->wheel_r = 0.33;
    P->k_susp = 35000.0;
    P->c_susp = 4000.0;
    P->rest_len = 0.3;
    /* R5: wheel spin inertia = 1/2 m_wheel r^2 s_inertia (App. F Tab. app_action_params) */
    P->wheel_inertia = 0.5 * 37.5 * 0.33 * 0.33 * 1.094;
    P->steer_inertia = 1.0;            /* R6                                                    */
    P->theta_max = 0.45;               /* App. F Tab. app_action_params                         */
    P->kp = 1839.5;
    P->kd = 110.5;
    P->tau_steer_max = 1200.0;
    P->tau_drive = 600.7;              /* R7: per front wheel (FWD, App. F)                     */
    P->tau_brk_f = 1090.5;
    P->tau_brk_r = 980.7;
    P->lambda_yaw = 10.6;              /* Sec. 3.2 yaw damping wrench                           */
    P->lambda_lat = 0.0;               /* R8: value not given                                   */
    P->u_z_min = 0.05;                 /* R12                                                   */
    P->k_contact = 1.0e6;              /* R20 */
    P->c_contact = 1.6e4;
    P->damp_ramp = 0.01;               /* R13b, R20: dampers ramp in over 1 cm          */
    P->wheelbase = 2.6;
    /* App. G Tab. app_reward_terms */
    P->goal_radius = 3.0;   P->w_goal = 45.0;  P->w_collision = 6.0;  P->w_crash = 10.0;
    P->w_lane_forb = 20.0;
    P->w_progress = 2.0;    P->progress_clip = 2.0;
    P->w_lane = 0.08;       P->lane_sigma = 1.75;  P->lane_wh = 0.8;
    P->w_offroad = 0.5;     P->offroad_lat = 3.25; P->offroad_dist = 6.0;
    P->w_idle = 0.05;       P->idle_speed = 1.0;
    P->ttc_alpha_v = 0.10;  P->ttc_pmax_v = 0.35;  P->ttc_floor = 0.5;  P->ttc_max = 10.0;
    P->ttc_alpha_e = 0.07;  P->ttc_pmax_e = 0.40;  P->edge_horizon = 40.0;
    P->drac_thresh = 3.4;   P->w_drac = 0.01;      P->drac_gap_floor = 0.1;   /* R26, R27 */
    P->drift_max = 100.0;   P->tilt_gz = -0.15;
    P->seg_gap_max = 3.0;   P->scene_half = 100.0; P->edge_half_width = 0.05; /* App. C */
    P->warmup_steps = 24;   P->max_steps = 1500;
    /* R28 */
    P->spawn_goal_min = 50.0; P->spawn_goal_max = 150.0;
    P->spawn_v_min = 5.0;     P->spawn_v_max = 20.0;
    P->spawn_spacing = 10.0;  P->park_x = 1000.0;  P->spawn_tries = 8;
    /* R9: friction table [precip][surface] */
    static const double mu[4][3] = {{0.90, 0.85, 0.60},
                                    {0.70, 0.65, 0.50},
                                    {0.50, 0.45, 0.40},
                                    {0.30, 0.25, 0.20}};
    memcpy(P->mu_table, mu, sizeof(mu));
    /* bicycle backend: the 30 degree steering limit of Sec. 4.4; accelerations
     * from the vehicle's actuator limits (App. F): 2 x 600.7 N m and
     * 2 x 1090.5 + 2 x 980.7 N m at r_w = 0.33 m on 1500 kg (a reading) */
    P->bike_theta_max = M_PI / 6.0;
    P->bike_a_drive = 2.0 * P->tau_drive / (P->wheel_r * P->mass);
    P->bike_a_brake = 2.0 * (P->tau_brk_f + P->tau_brk_r) / (P->wheel_r * P->mass);
    /* App. B: mu_static of the modified ALL model at 13.89 m/s, read off the
     * printed curves of Fig. friction_mu_vs_film (h = 0, 0.1, ..., 0.8 mm);
     * surface presets theta and T_d; the 1e-3 floor; Eq. weather_obs h_norm */
    static const double all_mu[3][9] = {
        {1.1048, 1.0657, 1.0161, 0.9593, 0.9039, 0.8595, 0.8302, 0.8134, 0.8044},   /* AC   */
        {1.2043, 1.1618, 1.1078, 1.0461, 0.9857, 0.9374, 0.9056, 0.8874, 0.8776},   /* SMA  */
        {1.3368, 1.2898, 1.2301, 1.1617, 1.0948, 1.0413, 1.0061, 0.9860, 0.9753}};  /* OGFC */
    memcpy(P->all_mu, all_mu, sizeof(all_mu));
    P->all_h_cut = 0.85;       /* F5: the figure's aquaplaning threshold */
    P->all_floor = 1e-3;
    P->all_theta[0] = 1.00; P->all_theta[1] = 1.09; P->all_theta[2] = 1.21;
    P->all_td[0] = 0.65;    P->all_td[1] = 0.80;    P->all_td[2] = 1.08;
    P->h_norm = 1.0;
    P->stribeck_b[0] = 4.8916; P->stribeck_b[1] = -7.91; P->stribeck_b[2] = 3.01; P->stribeck_b[3] = 3.40;
    P->weather_model = OR_WEATHER_TABLE;
}

uint64_t or_splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* ------------------------------------------------------------------ small vector helpers */
static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double a[3], const double b[3], double o[3]) {
    double x = a[1] * b[2] - a[2] * b[1];
    double y = a[2] * b[0] - a[0] * b[2];
    double z = a[0] * b[1] - a[1] * b[0];
    o[0] = x; o[1] = y; o[2] = z;
}
static double cross2(double ax, double ay, double bx, double by) { return ax * by - ay * bx; }
static double clampd(double x, double lo, double hi) { return x < lo ? lo : (x > hi ? hi : x); }

/* rotation matrix of a unit quaternion (w, x, y, z) */
static void quat_to_mat(const double* q, double R[3][3]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z);     R[0][2] = 2 * (x * z + w * y);
    R[1][0] = 2 * (x * y + w * z);     R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
    R[2][0] = 2 * (x * z - w * y);     R[2][1] = 2 * (y * z + w * x);     R[2][2] = 1 - 2 * (x * x + y * y);
}
static void mat_vec(const double R[3][3], const double v[3], double o[3]) {
    double x = R[0][0] * v[0] + R[0][1] * v[1] + R[0][2] * v[2];
    double y = R[1][0] * v[0] + R[1][1] * v[1] + R[1][2] * v[2];
    double z = R[2][0] * v[0] + R[2][1] * v[1] + R[2][2] * v[2];
    o[0] = x; o[1] = y; o[2] = z;
}

/* planar heading unit vector: the body x axis projected on the road plane */
static void heading_of(const double* f, double h[2]) {
    double R[3][3];
    quat_to_mat(f + OR_F_QW, R);
    double n = sqrt(R[0][0] * R[0][0] + R[1][0] * R[1][0]);
    if (n > 0) { h[0] = R[0][0] / n; h[1] = R[1][0] / n; }
    else { h[0] = 1; h[1] = 0; }
}

/* world vector -> ego frame (rotation by -psi) */
static void to_ego(const double h[2], double x, double y, double* bx, double* by) {
    *bx = h[0] * x + h[1] * y;
    *by = -h[1] * x + h[0] * y;
}

/* ------------------------------------------------------------------ roads */
static int poly_of_point(const or_scene* S, int w, int k) {
    int lo = S->poly_off[w], hi = S->poly_off[w + 1] - 1;
    while (lo < hi) { /* last polyline whose first point <= k */
        int mid = (lo + hi + 1) / 2;
        if (S->point_off[mid] <= k) lo = mid; else hi = mid - 1;
    }
    return lo;
}
static int is_lane(int t) { return t == 1 || t == 2; }
static int is_edge(int t) { return t == 15 || t == 16; }
static int in_box(const or_params* P, double x, double y) {
    return fabs(x) <= P->scene_half && fabs(y) <= P->scene_half;
}
/* segment k -> k+1 exists when both points are in polyline p, the gap is at most
 * seg_gap_max and both endpoints lie in the scene box (App. C "Segment generation") */
static int seg_valid(const or_params* P, const or_scene* S, int p, int k) {
    if (k + 1 >= S->point_off[p + 1]) return 0;
    double dx = S->px[k + 1] - S->px[k], dy = S->py[k + 1] - S->py[k];
    if (sqrt(dx * dx + dy * dy) > P->seg_gap_max) return 0;
    return in_box(P, S->px[k], S->py[k]) && in_box(P, S->px[k + 1], S->py[k + 1]);
}
/* road direction at point k: normalised (next - this) in its polyline; the last
 * point uses the previous segment; a one-point polyline has direction 0 */
static void point_dir(const or_scene* S, int p, int k, double d[2]) {
    int a, b;
    if (k + 1 < S->point_off[p + 1]) { a = k; b = k + 1; }
    else if (k - 1 >= S->point_off[p]) { a = k - 1; b = k; }
    else { d[0] = d[1] = 0; return; }
    double dx = S->px[b] - S->px[a], dy = S->py[b] - S->py[a];
    double n = sqrt(dx * dx + dy * dy);
    if (n > 0) { d[0] = dx / n; d[1] = dy / n; } else { d[0] = d[1] = 0; }
}
/* squared distance from q to segment a-b and the clamped parameter t */
static double seg_dist2(double ax, double ay, double bx, double by, double qx, double qy, double* t_out) {
    double ex = bx - ax, ey = by - ay;
    double l2 = ex * ex + ey * ey;
    double t = l2 > 0 ? ((qx - ax) * ex + (qy - ay) * ey) / l2 : 0.0;
    t = clampd(t, 0.0, 1.0);
    double dx = qx - ax - t * ex, dy = qy - ay - t * ey;
    if (t_out) *t_out = t;
    return dx * dx + dy * dy;
}

int or_nearest_lane(const or_params* P, const or_scene* S, int w, const double q[2], double* dist,
                    double* lateral, double tangent[2]) {
    int best = -1;
    double bd2 = INF_D;
    for (int p = S->poly_off[w]; p < S->poly_off[w + 1]; ++p) {
        if (!is_lane(S->poly_type[p])) continue;
        for (int k = S->point_off[p]; k < S->point_off[p + 1]; ++k) {
            if (!seg_valid(P, S, p, k)) continue;
            double d2 = seg_dist2(S->px[k], S->py[k], S->px[k + 1], S->py[k + 1], q[0], q[1], NULL);
            if (d2 < bd2) { bd2 = d2; best = k; }  /* ties: lowest index */
        }
    }
    if (best < 0) {
        if (dist) *dist = INF_D;
        if (lateral) *lateral = 0;
        if (tangent) tangent[0] = tangent[1] = 0;
        return -1;
    }
    double ex = S->px[best + 1] - S->px[best], ey = S->py[best + 1] - S->py[best];
    double n = sqrt(ex * ex + ey * ey);
    double tx = ex / n, ty = ey / n;
    if (dist) *dist = sqrt(bd2);
    if (lateral) *lateral = cross2(tx, ty, q[0] - S->px[best], q[1] - S->py[best]); /* left + */
    if (tangent) { tangent[0] = tx; tangent[1] = ty; }
    return best;
}

/* ------------------------------------------------------------------ pair geometry */
double or_sat(const or_params* P, const double ci[2], const double hi[2], const double cj[2],
              const double hj[2], double n_out[2]) {
    /* axes in the order (i.x, i.y, j.x, j.y); depth = minimum overlap, ties -> lowest axis */
    double ax[4][2] = {{hi[0], hi[1]}, {-hi[1], hi[0]}, {hj[0], hj[1]}, {-hj[1], hj[0]}};
    double dcx = cj[0] - ci[0], dcy = cj[1] - ci[1];
    double best = INF_D, sgn = 1.0;
    int bk = -1;
    for (int k = 0; k < 4; ++k) {
        double a0 = ax[k][0], a1 = ax[k][1];
        double ri = P->half_len * fabs(hi[0] * a0 + hi[1] * a1) + P->half_wid * fabs(-hi[1] * a0 + hi[0] * a1);
        double rj = P->half_len * fabs(hj[0] * a0 + hj[1] * a1) + P->half_wid * fabs(-hj[1] * a0 + hj[0] * a1);
        double d = dcx * a0 + dcy * a1;
        double o = ri + rj - fabs(d);
        if (o <= 0) { if (n_out) n_out[0] = n_out[1] = 0; return 0.0; }
        if (o < best) { best = o; bk = k; sgn = d >= 0 ? 1.0 : -1.0; }
    }
    if (n_out) { n_out[0] = sgn * ax[bk][0]; n_out[1] = sgn * ax[bk][1]; }
    return best;
}

/* F5: the printed mu_static(h) points joined linearly (0.1 mm apart); from
 * 0.8 mm linearly down to the floor at the aquaplaning threshold all_h_cut,
 * the floor beyond it (App. B: full grip loss for h >~ 0.85 mm, mu <= 1e-3 at
 * h >= 1.0 mm).  The film comes in hundredths of a millimetre, so the
 * interpolation weight r / 10 of the last step is exact. */
double or_all_mu_static(const or_params* P, int surface, int film_cmm) {
    const double* m = P->all_mu[surface];
    const int cut = (int)lround(P->all_h_cut * 100.0);
    if (film_cmm >= cut) return P->all_floor;
    if (film_cmm >= 80) return m[8] + (P->all_floor - m[8]) * (double)(film_cmm - 80) / (double)(cut - 80);
    const int k = film_cmm / 10, r = film_cmm % 10;
    return m[k] + (m[k + 1] - m[k]) * (double)r / 10.0;
}

/* Eq. app_stribeck_speed: v_s(h) = b1 exp(1000 b2 h + b3) + b4, h in metres */
double or_stribeck_vs(const or_params* P, double h_m) {
    const double* b = P->stribeck_b;
    return b[0] * exp(1000.0 * b[1] * h_m + b[2]) + b[3];
}

void or_ttc_circles(double L, double W, double WB, double* r, double* d) {
    /* App. D: r = max(0.45, 0.55 W), d = min(WB/2, max(0, L/2 - 0.8 r)) */
    double rr = fmax(0.45, 0.55 * W);
    *r = rr;
    *d = fmin(WB / 2.0, fmax(0.0, L / 2.0 - 0.8 * rr));
}

double or_ttc(const or_params* P, const double pi[2], const double hi[2], const double vi[2],
              const double pj[2], const double hj[2], const double vj[2]) {
    double r, d;
    or_ttc_circles(2 * P->half_len, 2 * P->half_wid, P->wheelbase, &r, &d);
    double bx, by;
    to_ego(hi, pj[0] - pi[0], pj[1] - pi[1], &bx, &by);
    if (bx < 0) return P->ttc_max;                 /* neighbour behind the ego */
    double dvx = vj[0] - vi[0], dvy = vj[1] - vi[1];
    double best = INF_D;
    for (int a = -1; a <= 1; ++a)
        for (int b = -1; b <= 1; ++b) {
            double dx = (pj[0] + b * d * hj[0]) - (pi[0] + a * d * hi[0]);
            double dy = (pj[1] + b * d * hj[1]) - (pi[1] + a * d * hi[1]);
            /* |dp + dv t|^2 = (2r)^2 : A t^2 + B t + C = 0 */
            double A = dvx * dvx + dvy * dvy;
            double B = 2 * (dx * dvx + dy * dvy);
            double C = dx * dx + dy * dy - 4 * r * r;
            double t;
            if (C <= 0) t = 0.0;                 /* circles already overlap */
            else if (B >= 0) continue;           /* separating: both roots <= 0 */
            else {
                double disc = B * B - 4 * A * C;
                if (disc < 0) continue;          /* closest approach misses */
                t = 2 * C / (-B + sqrt(disc));   /* smaller root, cancellation-free form */
            }
            if (t < best) best = t;
        }
    if (best >= INF_D) return P->ttc_max;
    return clampd(best, 0.0, P->ttc_max);
}

double or_drac(const or_params* P, const double pi[2], const double hi[2], const double vi[2], const double pj[2],
               const double hj[2], const double vj[2]) {
    double rx = pj[0] - pi[0], ry = pj[1] - pi[1];
    double dist = sqrt(rx * rx + ry * ry);
    if (!(dist > 0)) return 0.0;
    double ux = rx / dist, uy = ry / dist;
    double vr = -((vj[0] - vi[0]) * ux + (vj[1] - vi[1]) * uy);          /* closing speed */
    /* R26: the gap is the free distance along the line of centres: each
     * footprint reaches hl |h.u| + hw |h_perp.u| toward the other */
    double ei = P->half_len * fabs(hi[0] * ux + hi[1] * uy) + P->half_wid * fabs(-hi[1] * ux + hi[0] * uy);
    double ej = P->half_len * fabs(hj[0] * ux + hj[1] * uy) + P->half_wid * fabs(-hj[1] * ux + hj[0] * uy);
    double gap = fmax(dist - ei - ej, P->drac_gap_floor);
    return vr > 0 ? vr * vr / (2 * gap) : 0.0;
}

double or_lane_keep_q(const or_params* P, double lateral, double cos_dpsi) {
    double e = lateral / P->lane_sigma;
    return exp(-e * e) * ((1 - P->lane_wh) + P->lane_wh * fmax(0.0, cos_dpsi));
}

double or_penalty(double alpha, double tau, double tau_floor, double pmax) {
    return fmin(alpha / fmax(tau, tau_floor), pmax);
}

/* ------------------------------------------------------------------ one body substep */
static int alive(const int32_t* I, int a) { return (I[a * OR_NI + OR_I_STATUS] & OR_ALIVE) != 0; }

/* The substep of one chassis (R10 order): steering, suspension rays, predicted
 * velocities under gravity, springs, contact and damping, velocity-level
 * friction-circle impulses per wheel (Jacobi, shared by the wheels in contact),
 * brake, then positions and the quaternion. */
static void body_substep(const or_params* P, double* f, const double* act, const double Fc[2], double tau_c,
                         double h) {
    double thr = clampd(act[0], 0.0, 1.0);                       /* App. F: rectified throttle */
    double dstar = P->theta_max * clampd(act[1], -1.0, 1.0);    /* steering target          */
    double brk = clampd(act[2], 0.0, 1.0);                       /* rectified brake          */
    double mu = f[OR_F_MU];

    /* 1. steering PD (Eq. steer_pd), semi-implicit, angle clamped to +-theta_max (R11) */
    double tau_s = clampd(P->kp * (dstar - f[OR_F_DELTA]) - P->kd * f[OR_F_DDELTA], -P->tau_steer_max,
                          P->tau_steer_max);
    f[OR_F_DDELTA] += h * tau_s / P->steer_inertia;
    f[OR_F_DELTA] += h * f[OR_F_DDELTA];
    if (f[OR_F_DELTA] > P->theta_max) { f[OR_F_DELTA] = P->theta_max; f[OR_F_DDELTA] = 0; }
    if (f[OR_F_DELTA] < -P->theta_max) { f[OR_F_DELTA] = -P->theta_max; f[OR_F_DDELTA] = 0; }
    double delta = f[OR_F_DELTA];

    /* 2. rotation and world-frame inertia */
    double R[3][3];
    quat_to_mat(f + OR_F_QW, R);
    double Iinv[3][3], Iw[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double s = 0, t = 0;
            for (int k = 0; k < 3; ++k) {
                s += R[a][k] * R[b][k] / P->inertia[k];
                t += R[a][k] * R[b][k] * P->inertia[k];
            }
            Iinv[a][b] = s; Iw[a][b] = t;
        }
    double p[3] = {f[OR_F_PX], f[OR_F_PY], f[OR_F_PZ]};
    double v[3] = {f[OR_F_VX], f[OR_F_VY], f[OR_F_VZ]};
    double w[3] = {f[OR_F_WX], f[OR_F_WY], f[OR_F_WZ]};
    double u[3] = {R[0][2], R[1][2], R[2][2]};                /* body z axis in the world */

    /* 3. suspension rays along -u to the plane z = 0 */
    double N[4] = {0, 0, 0, 0}, rc[4][3];
    int hit[4] = {0, 0, 0, 0};
    for (int i = 0; i < 4; ++i) {
        double b[3] = {(i < 2 ? 1 : -1) * P->hard_x, (i % 2 == 0 ? 1 : -1) * P->hard_y, P->hard_z};
        double rb[3];
        mat_vec(R, b, rb);                                     /* hardpoint offset, world */
        double az = p[2] + rb[2];
        if (u[2] <= P->u_z_min) continue;                      /* R12 */
        double t = az / u[2];
        double l = t - P->wheel_r;
        if (l >= P->rest_len) continue;                        /* wheel off the ground */
        double x = P->rest_len - fmax(l, 0.0);                 /* R13 */
        double wr[3];
        cross3(w, rb, wr);
        double xdot = -(v[2] + wr[2]) / u[2];                  /* R14 */
        /* R13b: the damper engages over the first damp_ramp of compression, so
         * the normal force is continuous at touchdown */
        N[i] = fmax(0.0, P->k_susp * x + P->c_susp * xdot * fmin(1.0, x / P->damp_ramp));
        for (int k = 0; k < 3; ++k) rc[i][k] = rb[k] - t * u[k];   /* contact point - CoM */
        hit[i] = 1;
    }

    /* 4. predicted velocities: gravity, springs (+z), footprint contact, damping wrench */
    double F[3] = {Fc[0], Fc[1], -P->mass * P->g};
    double T[3] = {0, 0, tau_c - P->lambda_yaw * w[2]};
    if (P->lambda_lat != 0) {
        double ylat[3] = {R[0][1], R[1][1], R[2][1]};
        double vlat = dot3(v, ylat);
        for (int k = 0; k < 3; ++k) F[k] -= P->lambda_lat * vlat * ylat[k];
    }
    for (int i = 0; i < 4; ++i) {
        if (!hit[i]) continue;
        double fn[3] = {0, 0, N[i]}, tq[3];
        F[2] += N[i];
        cross3(rc[i], fn, tq);
        for (int k = 0; k < 3; ++k) T[k] += tq[k];
    }
    double Lw[3], gyro[3], net[3], dw[3];
    mat_vec(Iw, w, Lw);
    cross3(w, Lw, gyro);
    for (int k = 0; k < 3; ++k) net[k] = T[k] - gyro[k];
    mat_vec(Iinv, net, dw);
    double v1[3], w1[3];
    for (int k = 0; k < 3; ++k) { v1[k] = v[k] + h * F[k] / P->mass; w1[k] = w[k] + h * dw[k]; }
    double spin[4];
    for (int i = 0; i < 4; ++i)
        spin[i] = f[OR_F_S0 + i] + (i < 2 ? h * thr * P->tau_drive / P->wheel_inertia : 0.0);

    /* 5. friction impulses per wheel in contact, capped by the friction circle;
     * R16: the chassis share of every wheel's effective mass is that of one of
     * the four wheels, whichever are loaded (a Jacobi step relaxed by 1/4 never
     * overshoots and stays continuous when a wheel unloads) */
    const double nc = 4.0;
    double Pimp[3] = {0, 0, 0}, Limp[3] = {0, 0, 0};
    double spin2[4];
    for (int i = 0; i < 4; ++i) {
        spin2[i] = spin[i];
        if (!(N[i] > 0)) continue;
        double di = i < 2 ? delta : 0.0;
        double fb[3] = {cos(di), sin(di), 0}, fw[3];
        mat_vec(R, fb, fw);
        double fl = sqrt(fw[0] * fw[0] + fw[1] * fw[1]);
        if (!(fl > 0)) continue;
        double el[3] = {fw[0] / fl, fw[1] / fl, 0};
        double et[3] = {-el[1], el[0], 0};
        double wr[3], vc[3];
        cross3(w1, rc[i], wr);
        for (int k = 0; k < 3; ++k) vc[k] = v1[k] + wr[k];
        double rxe[3], tmp[3];
        cross3(rc[i], el, rxe);
        mat_vec(Iinv, rxe, tmp);
        double wl = P->wheel_r * P->wheel_r / P->wheel_inertia + nc * (1.0 / P->mass + dot3(rxe, tmp));
        cross3(rc[i], et, rxe);
        mat_vec(Iinv, rxe, tmp);
        double wt = nc * (1.0 / P->mass + dot3(rxe, tmp));
        double ul = spin[i] * P->wheel_r - dot3(vc, el);
        double ut = -dot3(vc, et);
        double jl = ul / wl, jt = ut / wt;
        double cap = mu * N[i] * h;
        double jn = sqrt(jl * jl + jt * jt);
        double s = jn <= cap ? 1.0 : cap / jn;                  /* R17 friction circle */
        jl *= s; jt *= s;
        double J[3] = {jl * el[0] + jt * et[0], jl * el[1] + jt * et[1], 0}, lj[3];
        cross3(rc[i], J, lj);
        for (int k = 0; k < 3; ++k) { Pimp[k] += J[k]; Limp[k] += lj[k]; }
        spin2[i] = spin[i] - jl * P->wheel_r / P->wheel_inertia;
    }
    /* brake: stick-slip soft threshold (R18) */
    for (int i = 0; i < 4; ++i) {
        double b = h * brk * (i < 2 ? P->tau_brk_f : P->tau_brk_r) / P->wheel_inertia;
        double m = fmax(fabs(spin2[i]) - b, 0.0);
        f[OR_F_S0 + i] = spin2[i] >= 0 ? m : -m;
    }

    /* 6. apply the impulses */
    double dwi[3];
    mat_vec(Iinv, Limp, dwi);
    for (int k = 0; k < 3; ++k) { v1[k] += Pimp[k] / P->mass; w1[k] += dwi[k]; }

    /* 7. positions and attitude: q += h/2 (0, w) (x) q, normalised */
    f[OR_F_PX] = p[0] + h * v1[0];
    f[OR_F_PY] = p[1] + h * v1[1];
    f[OR_F_PZ] = p[2] + h * v1[2];
    double qw = f[OR_F_QW], qx = f[OR_F_QX], qy = f[OR_F_QY], qz = f[OR_F_QZ];
    double dqw = -(w1[0] * qx + w1[1] * qy + w1[2] * qz);
    double dqx = w1[0] * qw + (w1[1] * qz - w1[2] * qy);
    double dqy = w1[1] * qw + (w1[2] * qx - w1[0] * qz);
    double dqz = w1[2] * qw + (w1[0] * qy - w1[1] * qx);
    qw += 0.5 * h * dqw; qx += 0.5 * h * dqx; qy += 0.5 * h * dqy; qz += 0.5 * h * dqz;
    double qn = sqrt(qw * qw + qx * qx + qy * qy + qz * qz);
    f[OR_F_QW] = qw / qn; f[OR_F_QX] = qx / qn; f[OR_F_QY] = qy / qn; f[OR_F_QZ] = qz / qn;
    f[OR_F_VX] = v1[0]; f[OR_F_VY] = v1[1]; f[OR_F_VZ] = v1[2];
    f[OR_F_WX] = w1[0]; f[OR_F_WY] = w1[1]; f[OR_F_WZ] = w1[2];
}

/* footprint contact of pair (i, j), i < j, at the current poses (R19, R20):
 * penalty force along the SAT normal, applied at the midpoint of the two
 * footprint centres in the plane of each CoM. */
static void pair_contact(const or_params* P, const double* fi, const double* fj, double Fi[2], double* Ti,
                         double Fj[2], double* Tj) {
    double ci[2] = {fi[OR_F_PX], fi[OR_F_PY]}, cj[2] = {fj[OR_F_PX], fj[OR_F_PY]};
    Fi[0] = Fi[1] = Fj[0] = Fj[1] = 0; *Ti = *Tj = 0;
    double dx = cj[0] - ci[0], dy = cj[1] - ci[1];
    double rcirc = 2 * sqrt(P->half_len * P->half_len + P->half_wid * P->half_wid);
    if (dx * dx + dy * dy > rcirc * rcirc) return;          /* bounding circles apart */
    double hi[2], hj[2], n[2];
    heading_of(fi, hi);
    heading_of(fj, hj);
    double depth = or_sat(P, ci, hi, cj, hj, n);
    if (!(depth > 0)) return;
    double vn = (fi[OR_F_VX] - fj[OR_F_VX]) * n[0] + (fi[OR_F_VY] - fj[OR_F_VY]) * n[1];
    double Fm = fmax(0.0, P->k_contact * depth + P->c_contact * vn * fmin(1.0, depth / P->damp_ramp));
    Fj[0] = Fm * n[0]; Fj[1] = Fm * n[1];
    Fi[0] = -Fj[0]; Fi[1] = -Fj[1];
    double mx = 0.5 * dx, my = 0.5 * dy;                      /* midpoint - ci ; midpoint - cj = -(m) */
    *Ti = cross2(mx, my, Fi[0], Fi[1]);
    *Tj = cross2(-mx, -my, Fj[0], Fj[1]);
}

void or_substep_world(const or_params* P, const or_scene* S, int w, double* F, const int32_t* I,
                      const double* actions, double h) {
    int a0 = S->agent_off[w], a1 = S->agent_off[w + 1], n = a1 - a0;
    if (n <= 0) return;
    double* fc = (double*)calloc((size_t)n * 3, sizeof(double));
    /* contact from the substep-start poses; pairs (i < j) in order */
    for (int i = 0; i < n; ++i) {
        if (!alive(I, a0 + i)) continue;
        for (int j = i + 1; j < n; ++j) {
            if (!alive(I, a0 + j)) continue;
            double Fi[2], Fj[2], Ti, Tj;
            pair_contact(P, F + (size_t)(a0 + i) * OR_NF, F + (size_t)(a0 + j) * OR_NF, Fi, &Ti, Fj, &Tj);
            fc[i * 3 + 0] += Fi[0]; fc[i * 3 + 1] += Fi[1]; fc[i * 3 + 2] += Ti;
            fc[j * 3 + 0] += Fj[0]; fc[j * 3 + 1] += Fj[1]; fc[j * 3 + 2] += Tj;
        }
    }
    for (int i = 0; i < n; ++i) {
        int a = a0 + i;
        if (!alive(I, a)) continue;
        body_substep(P, F + (size_t)a * OR_NF, actions + (size_t)a * 3, fc + i * 3, fc[i * 3 + 2], h);
    }
    free(fc);
}

/* ------------------------------------------------------------------ observation */
typedef struct { double key; int idx; } keyed;
static int cmp_keyed(const void* x, const void* y) {
    const keyed* a = (const keyed*)x;
    const keyed* b = (const keyed*)y;
    if (a->key < b->key) return -1;
    if (a->key > b->key) return 1;
    return (a->idx > b->idx) - (a->idx < b->idx);
}

/* K nearest alive other agents of agent a (XY distance, ties lowest index) */
static int knn_agents(const or_scene* S, int w, const double* F, const int32_t* I, int a, int* out) {
    int a0 = S->agent_off[w], a1 = S->agent_off[w + 1];
    keyed* buf = (keyed*)malloc(sizeof(keyed) * (size_t)(a1 - a0 + 1));
    int m = 0;
    for (int j = a0; j < a1; ++j) {
        if (j == a || !alive(I, j)) continue;
        double dx = F[(size_t)j * OR_NF + OR_F_PX] - F[(size_t)a * OR_NF + OR_F_PX];
        double dy = F[(size_t)j * OR_NF + OR_F_PY] - F[(size_t)a * OR_NF + OR_F_PY];
        buf[m].key = dx * dx + dy * dy; buf[m].idx = j; ++m;
    }
    qsort(buf, (size_t)m, sizeof(keyed), cmp_keyed);
    int k = m < OR_K_AGENTS ? m : OR_K_AGENTS;
    for (int t = 0; t < OR_K_AGENTS; ++t) out[t] = t < k ? buf[t].idx : -1;
    free(buf);
    return k;
}

static void observe_agent(const or_params* P, const or_scene* S, int w, const double* F, const int32_t* I, int a,
                          or_out* out) {
    double* o = out->obs ? out->obs + (size_t)a * OR_OBS : NULL;
    if (o) memset(o, 0, sizeof(double) * OR_OBS);
    if (out->lane_seg) out->lane_seg[a] = -1;
    if (out->knn_pts) for (int t = 0; t < OR_L_POINTS; ++t) out->knn_pts[(size_t)a * OR_L_POINTS + t] = -1;
    if (out->knn_agents) for (int t = 0; t < OR_K_AGENTS; ++t) out->knn_agents[(size_t)a * OR_K_AGENTS + t] = -1;
    if (!alive(I, a)) return;                                  /* parked agents see zeros */
    const double* f = F + (size_t)a * OR_NF;
    double hd[2];
    heading_of(f, hd);
    double p[2] = {f[OR_F_PX], f[OR_F_PY]};
    double v[2] = {f[OR_F_VX], f[OR_F_VY]};

    /* nearest driving lane (App. G), tangent oriented toward the goal (R22) */
    double dist, lat, tan2[2];
    int seg = or_nearest_lane(P, S, w, p, &dist, &lat, tan2);
    if (seg >= 0 && tan2[0] * (f[OR_F_GX] - p[0]) + tan2[1] * (f[OR_F_GY] - p[1]) < 0) {
        tan2[0] = -tan2[0]; tan2[1] = -tan2[1]; lat = -lat;
    }
    if (out->lane_seg) out->lane_seg[a] = seg;

    if (o) {
        /* ego group (App. D ego state + weather token, R24) */
        double gbx, gby, vbx, vby;
        to_ego(hd, f[OR_F_GX] - p[0], f[OR_F_GY] - p[1], &gbx, &gby);
        to_ego(hd, v[0], v[1], &vbx, &vby);
        double gn = sqrt(gbx * gbx + gby * gby);
        int pc = I[a * OR_NI + OR_I_PRECIP], sc = I[a * OR_NI + OR_I_SURFACE];
        o[0] = gbx / P->scene_half;
        o[1] = gby / P->scene_half;
        o[2] = gn > 0 ? gby / gn : 0.0;
        o[3] = gn > 0 ? gbx / gn : 1.0;
        o[4] = gn / P->scene_half;
        o[5] = vbx / 10.0;
        o[6] = vby / 10.0;
        /* weather token: (precip / 3, surface one-hot) of the table model, or
         * Eq. weather_obs (h / h_norm, one-hot AC, SMA, OGFC) of the ALL model */
        o[7] = P->weather_model == OR_WEATHER_ALL ? pc * 0.01 / P->h_norm : pc / 3.0;
        o[8] = sc == 0; o[9] = sc == 1; o[10] = sc == 2;
        o[11] = f[OR_F_WZ];
        o[12] = f[OR_F_DELTA] / P->theta_max;
        o[13] = f[OR_F_MU];
        o[14] = seg >= 0 ? lat / 3.6 : 0.0;
        o[15] = seg >= 0 ? cross2(tan2[0], tan2[1], hd[0], hd[1]) : 0.0;
    }

    /* K nearest agents with swept-circle TTC (App. D neighbour group, R23) */
    int nb[OR_K_AGENTS];
    knn_agents(S, w, F, I, a, nb);
    for (int t = 0; t < OR_K_AGENTS; ++t) {
        if (out->knn_agents) out->knn_agents[(size_t)a * OR_K_AGENTS + t] = nb[t];
        if (nb[t] < 0 || !o) continue;
        const double* g = F + (size_t)nb[t] * OR_NF;
        double hj[2];
        heading_of(g, hj);
        double pj[2] = {g[OR_F_PX], g[OR_F_PY]}, vj[2] = {g[OR_F_VX], g[OR_F_VY]};
        double bx, by, dvx, dvy;
        to_ego(hd, pj[0] - p[0], pj[1] - p[1], &bx, &by);
        to_ego(hd, vj[0] - v[0], vj[1] - v[1], &dvx, &dvy);
        double dpsi = atan2(cross2(hd[0], hd[1], hj[0], hj[1]), hd[0] * hj[0] + hd[1] * hj[1]);
        double* s = o + OR_EGO + t * OR_NBR_F;
        s[0] = bx / P->scene_half;
        s[1] = by / P->scene_half;
        s[2] = 2 * P->half_len / P->scene_half;
        s[3] = 2 * P->half_wid / P->scene_half;
        s[4] = dpsi / M_PI;
        s[5] = sqrt(vj[0] * vj[0] + vj[1] * vj[1]) / 10.0;
        s[6] = dvx / 10.0;
        s[7] = dvy / 10.0;
        s[8] = or_ttc(P, p, hd, v, pj, hj, vj) / P->ttc_max;
        s[9] = 1.0;
    }

    /* L nearest road points, all types (key: squared distance, ties lowest index) */
    int q0 = S->point_off[S->poly_off[w]], q1 = S->point_off[S->poly_off[w + 1]];
    keyed* buf = (keyed*)malloc(sizeof(keyed) * (size_t)(q1 - q0 + 1));
    int m = 0;
    for (int k = q0; k < q1; ++k) {
        double dx = S->px[k] - p[0], dy = S->py[k] - p[1];
        buf[m].key = dx * dx + dy * dy; buf[m].idx = k; ++m;
    }
    qsort(buf, (size_t)m, sizeof(keyed), cmp_keyed);
    int L = m < OR_L_POINTS ? m : OR_L_POINTS;
    for (int t = 0; t < L; ++t) {
        int k = buf[t].idx;
        if (out->knn_pts) out->knn_pts[(size_t)a * OR_L_POINTS + t] = k;
        if (!o) continue;
        int pl = poly_of_point(S, w, k);
        double d[2], bx, by, dbx, dby;
        point_dir(S, pl, k, d);
        to_ego(hd, S->px[k] - p[0], S->py[k] - p[1], &bx, &by);
        to_ego(hd, d[0], d[1], &dbx, &dby);
        int ty = S->poly_type[pl];
        double* s = o + OR_EGO + OR_K_AGENTS * OR_NBR_F + t * OR_PT_F;
        s[0] = bx / 10.0;
        s[1] = by / 10.0;
        s[2] = dbx;
        s[3] = dby;
        s[4] = ty / 20.0;
        s[5] = is_edge(ty);
        s[6] = 1.0;
    }
    free(buf);
}

void or_observe(const or_params* P, const or_scene* S, const double* F, const int32_t* I, or_out* out) {
    for (int w = 0; w < S->num_worlds; ++w)
        for (int a = S->agent_off[w]; a < S->agent_off[w + 1]; ++a) observe_agent(P, S, w, F, I, a, out);
}

/* ------------------------------------------------------------------ full observation (App. D) */
/* One agent's 1,929 values.  Road context: App. D selects the road points within
 * r = 10 m of the ego and orders them by their original polyline index; the points
 * are the segment midpoints baked at world build time (App. C "Segment generation",
 * "Metadata baking"), so the candidates are the world's valid segments k -> k+1 in
 * ascending k (polyline order, then point order), the test is |m - p|^2 <= r^2 on the
 * midpoint m, and the first 350 are kept.  Neighbours: the 24 nearest alive others
 * with self and dead agents at infinity (App. D). */
static void observe_full_agent(const or_params* P, const or_scene* S, int w, const double* F, const int32_t* I,
                               int a, double* o, int32_t* n_road, int32_t* n_veh, int32_t* road_idx,
                               int32_t* veh_idx) {
    if (o) memset(o, 0, sizeof(double) * OR_FULL_OBS);
    if (n_road) n_road[a] = 0;
    if (n_veh) n_veh[a] = 0;
    if (road_idx) for (int t = 0; t < OR_FULL_KR; ++t) road_idx[(size_t)a * OR_FULL_KR + t] = -1;
    if (veh_idx) for (int t = 0; t < OR_FULL_KV; ++t) veh_idx[(size_t)a * OR_FULL_KV + t] = -1;
    if (!alive(I, a)) return;
    const double* f = F + (size_t)a * OR_NF;
    double hd[2];
    heading_of(f, hd);
    double p[2] = {f[OR_F_PX], f[OR_F_PY]};
    double v[2] = {f[OR_F_VX], f[OR_F_VY]};

    /* ego group: App. D items 1-4, then the weather token analogue (four values) */
    if (o) {
        double gbx, gby, vbx, vby;
        to_ego(hd, f[OR_F_GX] - p[0], f[OR_F_GY] - p[1], &gbx, &gby);
        to_ego(hd, v[0], v[1], &vbx, &vby);
        double gn = sqrt(gbx * gbx + gby * gby);
        int pc = I[a * OR_NI + OR_I_PRECIP], sc = I[a * OR_NI + OR_I_SURFACE];
        o[0] = gbx / P->scene_half;
        o[1] = gby / P->scene_half;
        o[2] = gn > 0 ? gby / gn : 0.0;
        o[3] = gn > 0 ? gbx / gn : 1.0;
        o[4] = gn / P->scene_half;
        o[5] = vbx / 10.0;
        o[6] = vby / 10.0;
        /* weather token: (precip / 3, surface one-hot) of the table model, or
         * Eq. weather_obs (h / h_norm, one-hot AC, SMA, OGFC) of the ALL model */
        o[7] = P->weather_model == OR_WEATHER_ALL ? pc * 0.01 / P->h_norm : pc / 3.0;
        o[8] = sc == 0; o[9] = sc == 1; o[10] = sc == 2;
    }

    /* road context: every valid segment of the world, in index order */
    const double r = OR_FULL_RADIUS;
    int nr = 0;
    for (int pl = S->poly_off[w]; pl < S->poly_off[w + 1] && nr < OR_FULL_KR; ++pl) {
        for (int k = S->point_off[pl]; k < S->point_off[pl + 1] && nr < OR_FULL_KR; ++k) {
            if (!seg_valid(P, S, pl, k)) continue;
            double mx = 0.5 * (S->px[k] + S->px[k + 1]), my = 0.5 * (S->py[k] + S->py[k + 1]);
            double dx = mx - p[0], dy = my - p[1];
            if (dx * dx + dy * dy > r * r) continue;
            if (road_idx) road_idx[(size_t)a * OR_FULL_KR + nr] = k;
            if (o) {
                double ex = S->px[k + 1] - S->px[k], ey = S->py[k + 1] - S->py[k];
                double n = sqrt(ex * ex + ey * ey);
                double ux = n > 0 ? ex / n : 0.0, uy = n > 0 ? ey / n : 0.0;
                double bx, by, ubx, uby;
                to_ego(hd, dx, dy, &bx, &by);
                to_ego(hd, ux, uy, &ubx, &uby);
                double* s = o + OR_FULL_EGO + nr * OR_FULL_PT;
                s[0] = bx / r;
                s[1] = by / r;
                s[2] = S->poly_type[pl] / 20.0;
                s[3] = ubx;
                s[4] = uby;
            }
            ++nr;
        }
    }
    if (n_road) n_road[a] = nr;

    /* neighbour context: full sort of the alive others by (squared distance, index) */
    int a0 = S->agent_off[w], a1 = S->agent_off[w + 1];
    keyed* buf = (keyed*)malloc(sizeof(keyed) * (size_t)(a1 - a0 + 1));
    int m = 0;
    for (int j = a0; j < a1; ++j) {
        if (j == a || !alive(I, j)) continue;
        double dx = F[(size_t)j * OR_NF + OR_F_PX] - p[0], dy = F[(size_t)j * OR_NF + OR_F_PY] - p[1];
        buf[m].key = dx * dx + dy * dy; buf[m].idx = j; ++m;
    }
    qsort(buf, (size_t)m, sizeof(keyed), cmp_keyed);
    int nv = m < OR_FULL_KV ? m : OR_FULL_KV;
    for (int t = 0; t < nv; ++t) {
        int j = buf[t].idx;
        if (veh_idx) veh_idx[(size_t)a * OR_FULL_KV + t] = j;
        if (!o) continue;
        const double* g = F + (size_t)j * OR_NF;
        double hj[2];
        heading_of(g, hj);
        double pj[2] = {g[OR_F_PX], g[OR_F_PY]}, vj[2] = {g[OR_F_VX], g[OR_F_VY]};
        double bx, by;
        to_ego(hd, pj[0] - p[0], pj[1] - p[1], &bx, &by);
        double dpsi = atan2(cross2(hd[0], hd[1], hj[0], hj[1]), hd[0] * hj[0] + hd[1] * hj[1]);
        double* s = o + OR_FULL_EGO + OR_FULL_KR * OR_FULL_PT + t * OR_FULL_NB;
        s[0] = bx / P->scene_half;
        s[1] = by / P->scene_half;
        s[2] = 2 * P->half_len / P->scene_half;
        s[3] = 2 * P->half_wid / P->scene_half;
        s[4] = dpsi / M_PI;
        s[5] = sqrt(vj[0] * vj[0] + vj[1] * vj[1]) / 10.0;
        s[6] = or_ttc(P, p, hd, v, pj, hj, vj) / P->ttc_max;
    }
    free(buf);
    if (n_veh) n_veh[a] = nv;
}

void or_observe_full(const or_params* P, const or_scene* S, const double* F, const int32_t* I, double* obs,
                     int32_t* n_road, int32_t* n_veh, int32_t* road_idx, int32_t* veh_idx) {
    for (int w = 0; w < S->num_worlds; ++w)
        for (int a = S->agent_off[w]; a < S->agent_off[w + 1]; ++a)
            observe_full_agent(P, S, w, F, I, a, obs ? obs + (size_t)a * OR_FULL_OBS : NULL, n_road, n_veh,
                               road_idx, veh_idx);
}

/* ------------------------------------------------------------------ events and rewards */
static void events_agent(const or_params* P, const or_scene* S, int w, double* F, int32_t* I, int a,
                         const double prev[2], int flags, double* reward, uint32_t* ev, double* drac_out,
                         int32_t* lane_seg) {
    double* f = F + (size_t)a * OR_NF;
    int32_t* ii = I + (size_t)a * OR_NI;
    *reward = 0; *ev = 0; *drac_out = 0;
    if (lane_seg) *lane_seg = -1;
    ii[OR_I_STEP] += 1;
    double hd[2];
    heading_of(f, hd);
    double p[2] = {f[OR_F_PX], f[OR_F_PY]}, v[2] = {f[OR_F_VX], f[OR_F_VY]};
    double speed = sqrt(v[0] * v[0] + v[1] * v[1]);
    uint32_t e = 0;

    /* nearest lane: progress, lane keeping, off-road (App. G dense terms) */
    double dist, lat, tan2[2];
    int seg = or_nearest_lane(P, S, w, p, &dist, &lat, tan2);
    if (lane_seg) *lane_seg = seg;
    double r = 0;
    if (seg >= 0) {
        if (tan2[0] * (f[OR_F_GX] - p[0]) + tan2[1] * (f[OR_F_GY] - p[1]) < 0) {
            tan2[0] = -tan2[0]; tan2[1] = -tan2[1]; lat = -lat;
        }
        double prog = (p[0] - prev[0]) * tan2[0] + (p[1] - prev[1]) * tan2[1];
        r += P->w_progress * clampd(prog, -P->progress_clip, P->progress_clip);
        r += P->w_lane * or_lane_keep_q(P, lat, hd[0] * tan2[0] + hd[1] * tan2[1]);
    }
    if (fabs(lat) > P->offroad_lat || dist > P->offroad_dist) { e |= OR_EV_OFFROAD; r -= P->w_offroad; }
    if (speed < P->idle_speed) { e |= OR_EV_IDLE; r -= P->w_idle; }

    /* neighbours: TTC penalty, DRAC (R26), collision at the end-of-step poses */
    int nb[OR_K_AGENTS];
    knn_agents(S, w, F, I, a, nb);
    double tmin = P->ttc_max, dmax = 0;
    int n_nb = 0;
    for (int t = 0; t < OR_K_AGENTS; ++t) {
        if (nb[t] < 0) continue;
        ++n_nb;
        const double* g = F + (size_t)nb[t] * OR_NF;
        double hj[2];
        heading_of(g, hj);
        double pj[2] = {g[OR_F_PX], g[OR_F_PY]}, vj[2] = {g[OR_F_VX], g[OR_F_VY]};
        double tt = or_ttc(P, p, hd, v, pj, hj, vj);
        if (tt < tmin) tmin = tt;
        double dr = or_drac(P, p, hd, v, pj, hj, vj);
        if (dr > dmax) dmax = dr;
    }
    /* App. G: p(tau) of the minimum pairwise TTC over the neighbours, where a
     * neighbour behind the ego or on no collision course has TTC = tau_max
     * (App. D); so any neighbour costs at least alpha_v / tau_max = 0.01 per
     * step.  An agent without neighbours has no pairwise TTC and no term. */
    if (n_nb > 0) r -= or_penalty(P->ttc_alpha_v, tmin, P->ttc_floor, P->ttc_pmax_v);
    r -= P->w_drac * fmax(0.0, dmax - P->drac_thresh);
    *drac_out = dmax;
    if (dmax > f[OR_F_PEAK_DRAC]) f[OR_F_PEAK_DRAC] = dmax;

    int collided = 0;
    for (int j = S->agent_off[w]; j < S->agent_off[w + 1]; ++j) {
        if (j == a || !alive(I, j)) continue;
        const double* g = F + (size_t)j * OR_NF;
        double dx = g[OR_F_PX] - p[0], dy = g[OR_F_PY] - p[1];
        double rcirc = 2 * sqrt(P->half_len * P->half_len + P->half_wid * P->half_wid);
        if (dx * dx + dy * dy > rcirc * rcirc) continue;
        double hj[2], cj[2] = {g[OR_F_PX], g[OR_F_PY]};
        heading_of(g, hj);
        if (or_sat(P, p, hd, cj, hj, NULL) > 0) { collided = 1; break; }
    }
    if (collided && ii[OR_I_STEP] > P->warmup_steps) e |= OR_EV_COLLISION;

    /* road edges: lane-forbidden (three circles vs edge segments), edge TTC (R25) */
    double rc, dc;
    or_ttc_circles(2 * P->half_len, 2 * P->half_wid, P->wheelbase, &rc, &dc);
    double tedge = INF_D;
    int forb = 0;
    for (int pl = S->poly_off[w]; pl < S->poly_off[w + 1]; ++pl) {
        if (!is_edge(S->poly_type[pl])) continue;
        for (int k = S->point_off[pl]; k < S->point_off[pl + 1]; ++k) {
            if (!seg_valid(P, S, pl, k)) continue;
            double ax = S->px[k], ay = S->py[k], bx = S->px[k + 1], by = S->py[k + 1];
            for (int c = -1; c <= 1; ++c) {
                double cx = p[0] + c * dc * hd[0], cy = p[1] + c * dc * hd[1];
                double lim = rc + P->edge_half_width;
                if (seg_dist2(ax, ay, bx, by, cx, cy, NULL) < lim * lim) forb = 1;
            }
            double ex = bx - ax, ey = by - ay;
            double den = cross2(v[0], v[1], ex, ey);
            if (den != 0) {
                double t = cross2(ax - p[0], ay - p[1], ex, ey) / den;
                double s = cross2(ax - p[0], ay - p[1], v[0], v[1]) / den;
                if (t >= 0 && s >= 0 && s <= 1 && speed * t <= P->edge_horizon && t < tedge) tedge = t;
            }
        }
    }
    if (tedge < INF_D) r -= or_penalty(P->ttc_alpha_e, tedge, P->ttc_floor, P->ttc_pmax_e);
    if (forb) e |= OR_EV_LANE_FORB;

    /* goal and crash (App. G sparse terms) */
    double gx = f[OR_F_GX] - p[0], gy = f[OR_F_GY] - p[1];
    if (sqrt(gx * gx + gy * gy) <= P->goal_radius) e |= OR_EV_GOAL;
    double R[3][3];
    quat_to_mat(f + OR_F_QW, R);
    double sx = p[0] - f[OR_F_SX], sy = p[1] - f[OR_F_SY];
    if (f[OR_F_PZ] < 0 || sqrt(sx * sx + sy * sy) > P->drift_max || -R[2][2] > P->tilt_gz) e |= OR_EV_CRASH;

    /* the four sparse events are mutually exclusive: the first one in the
     * order goal, collision, crash, lane-forbidden delivers its reward */
    if (e & OR_EV_GOAL) r += P->w_goal;
    else if (e & OR_EV_COLLISION) r -= P->w_collision;
    else if (e & OR_EV_CRASH) r -= P->w_crash;
    else if (e & OR_EV_LANE_FORB) r -= P->w_lane_forb;
    if (ii[OR_I_STEP] >= P->max_steps) e |= OR_EV_TIMEOUT;
    *reward = r;
    *ev = e;
    (void)flags;
}

void or_events(const or_params* P, const or_scene* S, double* F, int32_t* I, const double* prev_xy, int flags,
               or_out* out) {
    int A = S->agent_off[S->num_worlds];
    double* drac = (double*)calloc((size_t)A + 1, sizeof(double));
    /* every agent's events read the end-of-step state of all agents before any
     * peak-DRAC update is visible; peak DRAC is not read by events, so the
     * in-place update is order independent */
    for (int w = 0; w < S->num_worlds; ++w)
        for (int a = S->agent_off[w]; a < S->agent_off[w + 1]; ++a) {
            double r = 0; uint32_t e = 0; int32_t ls = -1;
            if (alive(I, a)) events_agent(P, S, w, F, I, a, prev_xy + 2 * (size_t)a, flags, &r, &e, &drac[a], &ls);
            if (out->reward) out->reward[a] = r;
            if (out->events) out->events[a] = e;
            if (out->drac) out->drac[a] = drac[a];
            if (out->lane_seg) out->lane_seg[a] = ls;
        }
    free(drac);
}

/* ------------------------------------------------------------------ placement and resets */
void or_place_agent(const or_params* P, double* F, int32_t* I, int a, double x, double y, double psi, double v0,
                    double gx, double gy, int precip, int surface) {
    double* f = F + (size_t)a * OR_NF;
    int32_t* ii = I + (size_t)a * OR_NI;
    double c = cos(psi), s = sin(psi);
    f[OR_F_PX] = x; f[OR_F_PY] = y;
    /* static equilibrium: four springs carry m g, compression m g / (4 k) */
    f[OR_F_PZ] = -P->hard_z + (P->rest_len - P->mass * P->g / (4 * P->k_susp)) + P->wheel_r;
    f[OR_F_QW] = cos(0.5 * psi); f[OR_F_QX] = 0; f[OR_F_QY] = 0; f[OR_F_QZ] = sin(0.5 * psi);
    f[OR_F_VX] = v0 * c; f[OR_F_VY] = v0 * s; f[OR_F_VZ] = 0;
    f[OR_F_WX] = f[OR_F_WY] = f[OR_F_WZ] = 0;
    for (int i = 0; i < 4; ++i) f[OR_F_S0 + i] = v0 / P->wheel_r;  /* rolling wheels */
    f[OR_F_DELTA] = 0; f[OR_F_DDELTA] = 0;
    f[OR_F_GX] = gx; f[OR_F_GY] = gy;
    f[OR_F_SX] = x; f[OR_F_SY] = y;
    f[OR_F_MU] = P->weather_model == OR_WEATHER_ALL ? or_all_mu_static(P, surface, precip)
                                                   : P->mu_table[precip][surface];
    f[OR_F_PEAK_DRAC] = 0;
    ii[OR_I_PRECIP] = precip; ii[OR_I_SURFACE] = surface;
    ii[OR_I_STEP] = 0;
    ii[OR_I_STATUS] = OR_ALIVE;
}

static void park_agent(const or_params* P, double* F, int32_t* I, int a) {
    double* f = F + (size_t)a * OR_NF;
    /* App. G: terminated agents are teleported off stage to x = 1000 m */
    f[OR_F_PX] = P->park_x; f[OR_F_PY] = 0;
    f[OR_F_VX] = f[OR_F_VY] = f[OR_F_VZ] = 0;
    f[OR_F_WX] = f[OR_F_WY] = f[OR_F_WZ] = 0;
    for (int i = 0; i < 4; ++i) f[OR_F_S0 + i] = 0;
    I[a * OR_NI + OR_I_STATUS] = OR_PARKED;
}

/* counter-based draw j of attempt r of episode e of agent a (R28) */
static uint64_t draw(uint64_t seed, int a, int e, int r, int j) {
    uint64_t h = or_splitmix64(or_splitmix64(seed) ^ (uint64_t)(uint32_t)a);
    return or_splitmix64(h ^ (((uint64_t)(uint32_t)e << 32) | (uint64_t)(uint32_t)(r * 4 + j)));
}
static double u24(uint64_t h) { return (double)(h >> 40) * (1.0 / 16777216.0); }

/* arc length from the first point of polyline p to point k */
static double arc_to(const or_scene* S, int p, int k) {
    double s = 0;
    for (int i = S->point_off[p]; i < k; ++i) {
        double dx = S->px[i + 1] - S->px[i], dy = S->py[i + 1] - S->py[i];
        s += sqrt(dx * dx + dy * dy);
    }
    return s;
}

/* spawn candidates of world w: lane points with at least spawn_goal_min of lane ahead;
 * if there is none, every lane point */
static int spawn_candidates(const or_params* P, const or_scene* S, int w, int* out) {
    int m = 0;
    for (int pass = 0; pass < 2 && m == 0; ++pass)
        for (int p = S->poly_off[w]; p < S->poly_off[w + 1]; ++p) {
            if (!is_lane(S->poly_type[p])) continue;
            int k1 = S->point_off[p + 1];
            double total = arc_to(S, p, k1 - 1);
            for (int k = S->point_off[p]; k < k1; ++k)
                if (pass == 1 || total - arc_to(S, p, k) >= P->spawn_goal_min) out[m++] = k;
        }
    return m;
}

static void respawn_world(const or_params* P, const or_scene* S, int w, double* F, int32_t* I, const uint8_t* mask,
                          uint64_t seed) {
    int a0 = S->agent_off[w], a1 = S->agent_off[w + 1];
    int q0 = S->point_off[S->poly_off[w]], q1 = S->point_off[S->poly_off[w + 1]];
    int* cand = (int*)malloc(sizeof(int) * (size_t)(q1 - q0 + 1));
    int nc = spawn_candidates(P, S, w, cand);
    for (int a = a0; a < a1; ++a) {
        if (!mask[a]) continue;
        int ep = I[a * OR_NI + OR_I_EPISODE] + 1;
        double bx = 0, by = 0, bpsi = 0, bv = P->spawn_v_min, bgx = P->spawn_goal_min, bgy = 0, bscore = -1;
        for (int r = 0; r < P->spawn_tries; ++r) {
            /* R28b: a world without lane points spawns slot k at (0, k * spacing),
             * heading +x, goal spawn_goal_min ahead */
            double x = 0, y = (a - a0) * P->spawn_spacing, psi = 0, gx = P->spawn_goal_min, gy = y;
            if (nc > 0) {
                int k = cand[(uint32_t)(draw(seed, a, ep, r, 0) >> 32) % (uint32_t)nc];
                int p = poly_of_point(S, w, k);
                double d[2];
                point_dir(S, p, k, d);
                x = S->px[k]; y = S->py[k];
                psi = atan2(d[1], d[0]);
                double dg = P->spawn_goal_min + (P->spawn_goal_max - P->spawn_goal_min) * u24(draw(seed, a, ep, r, 1));
                int k1 = S->point_off[p + 1], g = k1 - 1;
                double s = 0;
                for (int j = k + 1; j < k1; ++j) {
                    double dx = S->px[j] - S->px[j - 1], dy = S->py[j] - S->py[j - 1];
                    s += sqrt(dx * dx + dy * dy);
                    if (s >= dg) { g = j; break; }
                }
                gx = S->px[g]; gy = S->py[g];
            }
            double v0 = P->spawn_v_min + (P->spawn_v_max - P->spawn_v_min) * u24(draw(seed, a, ep, r, 2));
            /* spacing: distance to every other alive agent of the world that is not
             * waiting to respawn after this one */
            double dmin = INF_D;
            for (int j = a0; j < a1; ++j) {
                if (j == a || !alive(I, j)) continue;
                if (j > a && mask[j]) continue;
                double dx = F[(size_t)j * OR_NF + OR_F_PX] - x, dy = F[(size_t)j * OR_NF + OR_F_PY] - y;
                double d2 = dx * dx + dy * dy;
                if (d2 < dmin) dmin = d2;
            }
            if (dmin > bscore) { bscore = dmin; bx = x; by = y; bpsi = psi; bv = v0; bgx = gx; bgy = gy; }
            if (dmin >= P->spawn_spacing * P->spawn_spacing) break;
        }
        int pc = I[a * OR_NI + OR_I_PRECIP], sc = I[a * OR_NI + OR_I_SURFACE];
        or_place_agent(P, F, I, a, bx, by, bpsi, bv, bgx, bgy, pc, sc);
        I[a * OR_NI + OR_I_EPISODE] = ep;
    }
    free(cand);
}

void or_reset(const or_params* P, const or_scene* S, double* F, int32_t* I, const uint8_t* mask, uint64_t seed,
              or_out* out) {
    for (int w = 0; w < S->num_worlds; ++w) respawn_world(P, S, w, F, I, mask, seed);
    int A = S->agent_off[S->num_worlds];
    for (int a = 0; a < A; ++a)
        if (mask[a]) I[a * OR_NI + OR_I_EVENTS] = OR_EV_RESPAWNED;
    or_observe(P, S, F, I, out);
}

static int finite_state(const double* f) {
    for (int k = 0; k < OR_NF; ++k) if (!isfinite(f[k])) return 0;
    return 1;
}

void or_bicycle_agent(const or_params* P, double* f, const double* act, double dt) {
    double thr = clampd(act[0], 0.0, 1.0), brk = clampd(act[2], 0.0, 1.0);
    double delta = P->bike_theta_max * clampd(act[1], -1.0, 1.0);
    double lr = 0.5 * P->wheelbase;
    double beta = atan(0.5 * tan(delta));
    double psi = 2.0 * atan2(f[OR_F_QZ], f[OR_F_QW]);
    double v = sqrt(f[OR_F_VX] * f[OR_F_VX] + f[OR_F_VY] * f[OR_F_VY]);
    double a = P->bike_a_drive * thr - P->bike_a_brake * brk;
    double v1 = fmax(0.0, v + a * dt);
    double r = v1 / lr * sin(beta);
    f[OR_F_PX] += v1 * cos(psi + beta) * dt;
    f[OR_F_PY] += v1 * sin(psi + beta) * dt;
    double psi1 = psi + r * dt;
    f[OR_F_PZ] = -P->hard_z + (P->rest_len - P->mass * P->g / (4 * P->k_susp)) + P->wheel_r;
    f[OR_F_QW] = cos(0.5 * psi1); f[OR_F_QX] = 0; f[OR_F_QY] = 0; f[OR_F_QZ] = sin(0.5 * psi1);
    f[OR_F_VX] = v1 * cos(psi1 + beta); f[OR_F_VY] = v1 * sin(psi1 + beta); f[OR_F_VZ] = 0;
    f[OR_F_WX] = 0; f[OR_F_WY] = 0; f[OR_F_WZ] = r;
    for (int i = 0; i < 4; ++i) f[OR_F_S0 + i] = v1 / P->wheel_r;
    f[OR_F_DELTA] = delta; f[OR_F_DDELTA] = 0;
}

int or_step(const or_params* P, const or_scene* S, double* F, int32_t* I, const double* actions, double dt,
            int substeps, uint64_t seed, int flags, or_out* out) {
    int A = S->agent_off[S->num_worlds];
    double h = dt / substeps;
    double* prev = (double*)malloc(sizeof(double) * 2 * (size_t)A + 16);
    uint8_t* mask = (uint8_t*)calloc((size_t)A + 1, 1);
    double* rew = (double*)calloc((size_t)A + 1, sizeof(double));
    uint32_t* ev = (uint32_t*)calloc((size_t)A + 1, sizeof(uint32_t));
    int bad = 0;
    for (int a = 0; a < A; ++a) {
        prev[2 * a] = F[(size_t)a * OR_NF + OR_F_PX];
        prev[2 * a + 1] = F[(size_t)a * OR_NF + OR_F_PY];
    }
    if (flags & OR_FLAG_BICYCLE) {
        for (int a = 0; a < A; ++a)
            if (alive(I, a)) or_bicycle_agent(P, F + (size_t)a * OR_NF, actions + 3 * (size_t)a, dt);
    } else {
        for (int w = 0; w < S->num_worlds; ++w)
            for (int s = 0; s < substeps; ++s) or_substep_world(P, S, w, F, I, actions, h);
    }
    /* non-finite guard: such agents leave the world before events are computed */
    uint8_t* nonfin = (uint8_t*)calloc((size_t)A + 1, 1);
    for (int a = 0; a < A; ++a)
        if (alive(I, a) && !finite_state(F + (size_t)a * OR_NF)) {
            nonfin[a] = 1; ++bad;
            park_agent(P, F, I, a);
        }
    or_out ev_out = {0};
    ev_out.reward = rew; ev_out.events = ev; ev_out.drac = out ? out->drac : NULL;
    or_events(P, S, F, I, prev, flags, &ev_out);
    for (int a = 0; a < A; ++a) {
        if (nonfin[a]) { ev[a] = OR_EV_NONFINITE; rew[a] = 0; }
        uint32_t sparse = OR_EV_GOAL | OR_EV_COLLISION | OR_EV_CRASH | OR_EV_LANE_FORB;
        int term = nonfin[a] || (!(flags & OR_FLAG_INVINCIBLE) && (ev[a] & sparse));
        int done = term || (ev[a] & OR_EV_TIMEOUT);
        if (out && out->done) out->done[a] = (uint8_t)done;
        if (done) {
            if (flags & OR_FLAG_AUTO_RESET) mask[a] = 1;
            else if (!nonfin[a]) park_agent(P, F, I, a);
        }
    }
    if (flags & OR_FLAG_AUTO_RESET)
        for (int w = 0; w < S->num_worlds; ++w) respawn_world(P, S, w, F, I, mask, seed);
    for (int a = 0; a < A; ++a) {
        if (mask[a]) ev[a] |= OR_EV_RESPAWNED;
        I[a * OR_NI + OR_I_EVENTS] = (int32_t)ev[a];
        if (out && out->reward) out->reward[a] = rew[a];
        if (out && out->events) out->events[a] = ev[a];
    }
    if (out) {
        or_out ob = *out;
        ob.reward = NULL; ob.done = NULL; ob.events = NULL; ob.drac = NULL;
        or_observe(P, S, F, I, &ob);
    }
    free(prev); free(mask); free(rew); free(ev); free(nonfin);
    return bad;
}
