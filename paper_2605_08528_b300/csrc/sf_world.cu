// sf_world.cu -- the fused per-world kernel of the vehicle step (sm_103a).
//
// One warp steps one world: lane l owns agent (first agent of the world + l),
// so a world holds at most 32 agents.  Every substep the lanes publish their
// footprint (centre, heading, velocity) in shared memory, each lane sums the
// penalty contact of every overlapping pair it belongs to (pairs evaluated in
// canonical (lo, hi) order so both partners see bit-identical forces), then
// integrates its own chassis.  After the substeps the warp computes events and
// rewards from the end-of-step poses, respawns done agents one after another
// (the spacing test is a warp-wide min over the other agents), and writes the
// observations.  All road queries scan the world's points in ascending index
// order, so every selection (nearest segment, k nearest points / agents) is the
// lexicographic (key, index) minimum.
//
// The model follows SceneFactory (arXiv 2605.08528): steering PD (Sec. 3.2
// Eq. steer_pd), FWD drive and 4-wheel brakes (App. F), rectified throttle and
// brake (App. F), yaw damping wrench (Sec. 3.2), rewards and events (App. G),
// observations (App. D), teleport resets (App. J).  The tire/suspension/contact
// model is the raycast, friction-circle, symplectic-Euler reading of the
// unstated PhysX internals.
#include "sf_internal.cuh"

#include <math.h>

using namespace sfk;

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
#define kInf __int_as_float(0x7f800000)

struct Agent {
    float px, py, pz, dl;
    float dpx, dpy, dpz;   // displacement since the start of the control step
    float qw, qx, qy, qz;
    float vx, vy, vz, dd;
    float wx, wy, wz, mu;
    float s0, s1, s2, s3;
    float gx, gy, sx, sy;
    float peak;
    uint32_t meta;
    int step, episode;
};

__device__ __forceinline__ float clampf(float x, float lo, float hi) { return x < lo ? lo : (x > hi ? hi : x); }
// a*b + c*d rounded one fixed way (c*d rounded, then one fused multiply-add):
// the step's kernels inline the same geometry in different contexts, and a
// contraction left to the compiler could round them differently
__device__ __forceinline__ float dot2(float a, float b, float c, float d) { return __fmaf_rn(a, b, __fmul_rn(c, d)); }
__device__ __forceinline__ float norm2(float x, float y) { return dot2(x, x, y, y); }
__device__ __forceinline__ float cross2(float ax, float ay, float bx, float by) { return dot2(ax, by, -ay, bx); }
// named barrier `id` over n threads (a multiple of 32): arrive without waiting / wait
__device__ __forceinline__ void named_bar_arrive(int id, int n) { asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory"); }
__device__ __forceinline__ void named_bar_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }
__device__ __forceinline__ uint32_t status_of(uint32_t meta) { return (meta >> 16) & 0xFFu; }
__device__ __forceinline__ uint32_t with_status(uint32_t meta, uint32_t st) { return (meta & 0xFFFFu) | (st << 16); }

// SplitMix64 (Steele, Lea, Flood 2014): the counter-based generator of resets.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
    unsigned long long z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ unsigned long long reset_draw(unsigned long long seed, int a, int e, int r, int j) {
    unsigned long long h = splitmix64(splitmix64(seed) ^ (unsigned long long)(uint32_t)a);
    return splitmix64(h ^ (((unsigned long long)(uint32_t)e << 32) | (unsigned long long)(uint32_t)(r * 4 + j)));
}
__device__ __forceinline__ float u24(unsigned long long h) { return (float)(uint32_t)(h >> 40) * (1.0f / 16777216.0f); }


__device__ __forceinline__ void quat_to_mat(float w, float x, float y, float z, float R[3][3]) {
    R[0][0] = 1.f - 2.f * (y * y + z * z); R[0][1] = 2.f * (x * y - w * z);       R[0][2] = 2.f * (x * z + w * y);
    R[1][0] = 2.f * (x * y + w * z);       R[1][1] = 1.f - 2.f * (x * x + z * z); R[1][2] = 2.f * (y * z - w * x);
    R[2][0] = 2.f * (x * z - w * y);       R[2][1] = 2.f * (y * z + w * x);       R[2][2] = 1.f - 2.f * (x * x + y * y);
}

// planar heading: body x axis projected on the road plane
__device__ __forceinline__ void heading_of(float qw, float qx, float qy, float qz, float& hx, float& hy) {
    float r00 = 1.f - 2.f * (qy * qy + qz * qz);
    float r10 = 2.f * (qx * qy + qw * qz);
    const float n2 = norm2(r00, r10);
    if (n2 > 0.f) {
        const float rn = rsqrtf(n2);
        hx = __fmul_rn(r00, rn); hy = __fmul_rn(r10, rn);
    } else {
        hx = 1.f; hy = 0.f;
    }
}

__device__ __forceinline__ void to_ego(float hx, float hy, float x, float y, float& bx, float& by) {
    bx = dot2(hx, x, hy, y);
    by = dot2(hx, y, -hy, x);
}

__device__ __forceinline__ float seg_dist2(float ax, float ay, float bx, float by, float qx, float qy) {
    float ex = bx - ax, ey = by - ay;
    float l2 = norm2(ex, ey);
    float t = l2 > 0.f ? dot2(qx - ax, ex, qy - ay, ey) / l2 : 0.f;
    t = clampf(t, 0.f, 1.f);
    float dx = __fmaf_rn(-t, ex, qx - ax), dy = __fmaf_rn(-t, ey, qy - ay);
    return norm2(dx, dy);
}

// ------------------------------------------------------------------ footprint contact
// 2-D SAT of two 4.5 x 1.8 m footprints; axes (i.x, i.y, j.x, j.y); depth is the
// minimum overlap (ties: lowest axis), normal oriented from i to j.
__device__ __forceinline__ float sat2d(float cix, float ciy, float hix, float hiy, float cjx, float cjy, float hjx,
                                       float hjy, float& nx, float& ny) {
    const float ax[4] = {hix, -hiy, hjx, -hjy};
    const float ay[4] = {hiy, hix, hjy, hjx};
    float dcx = cjx - cix, dcy = cjy - ciy;
    float best = kInf, sgn = 1.f;
    int bk = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float a0 = ax[k], a1 = ay[k];
        float ri = kHalfLen * fabsf(hix * a0 + hiy * a1) + kHalfWid * fabsf(-hiy * a0 + hix * a1);
        float rj = kHalfLen * fabsf(hjx * a0 + hjy * a1) + kHalfWid * fabsf(-hjy * a0 + hjx * a1);
        float d = dcx * a0 + dcy * a1;
        float o = ri + rj - fabsf(d);
        if (o <= 0.f) { nx = ny = 0.f; return 0.f; }
        if (o < best) { best = o; bk = k; sgn = d >= 0.f ? 1.f : -1.f; }
    }
    float bx = bk == 0 ? ax[0] : bk == 1 ? ax[1] : bk == 2 ? ax[2] : ax[3];
    float by = bk == 0 ? ay[0] : bk == 1 ? ay[1] : bk == 2 ? ay[2] : ay[3];
    nx = sgn * bx; ny = sgn * by;
    return best;
}

// penalty force of pair (lo, hi) on hi, and the torque both bodies receive
// (force pair at the midpoint of the footprint centres, in each CoM plane)
// (ci, di): start-of-step position and in-step displacement of each agent; the
// separation (cj - ci) + (dj - di) avoids rounding the positions of every substep
__device__ __forceinline__ void pair_force(float cix, float ciy, float dix, float diy, float hix, float hiy, float vix,
                                           float viy, float cjx, float cjy, float djx, float djy, float hjx, float hjy,
                                           float vjx, float vjy, float& fx, float& fy, float& tz) {
    fx = fy = tz = 0.f;
    float dx = (cjx - cix) + (djx - dix), dy = (cjy - ciy) + (djy - diy);
    if (dx * dx + dy * dy > kPairCull2) return;
    float nx, ny;
    float depth = sat2d(0.f, 0.f, hix, hiy, dx, dy, hjx, hjy, nx, ny);
    if (!(depth > 0.f)) return;
    float vn = (vix - vjx) * nx + (viy - vjy) * ny;
    float fm = fmaxf(0.f, kKContact * depth + kCContact * vn * fminf(1.f, depth / kDampRamp));
    fx = fm * nx; fy = fm * ny;
    float mx = 0.5f * dx, my = 0.5f * dy;
    tz = cross2(-mx, -my, fx, fy);
}

// ------------------------------------------------------------------ one chassis substep
// steering PD, suspension rays, predicted velocities, friction-circle wheel
// impulses (Jacobi, shared by the wheels in contact), brake, positions.
// steering PD (Eq. steer_pd), semi-implicit, angle clamped: decoupled from the chassis
__device__ __forceinline__ void steer_substep(Agent& A, float dstar, float h) {
    float ts = clampf(kKp * (dstar - A.dl) - kKd * A.dd, -kTauSteer, kTauSteer);
    A.dd += h * ts / kSteerI;
    A.dl += h * A.dd;
    if (A.dl > kThetaMax) { A.dl = kThetaMax; A.dd = 0.f; }
    if (A.dl < -kThetaMax) { A.dl = -kThetaMax; A.dd = 0.f; }
}

__device__ __forceinline__ void body_substep(Agent& A, float thr, float dstar, float brk, float fcx, float fcy,
                                             float tcz, float h) {
    // 1. steering
    steer_substep(A, dstar, h);

    // 2. rotation, world inverse inertia (symmetric)
    float R[3][3];
    quat_to_mat(A.qw, A.qx, A.qy, A.qz, R);
    float Ii[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            Ii[a][b] = R[a][0] * R[b][0] * kInvIxx + R[a][1] * R[b][1] * kInvIyy + R[a][2] * R[b][2] * kInvIzz;
    const float ux = R[0][2], uy = R[1][2], uz = R[2][2];
    const float inv_uz = uz > kUzMin ? 1.f / uz : 0.f;   // shared by the four rays

    // 3. suspension rays from the hardpoints along -u to the plane z = 0.  The
    // four wheels are computed without branches and a wheel whose ray misses
    // selects zeros, so that the wheels' dependency chains interleave
    float N[4], rcx[4], rcy[4], rcz[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float bx = i < 2 ? kHardX : -kHardX;
        const float by = (i & 1) == 0 ? kHardY : -kHardY;
        const float bz = kHardZ;
        float rbx = R[0][0] * bx + R[0][1] * by + R[0][2] * bz;
        float rby = R[1][0] * bx + R[1][1] * by + R[1][2] * bz;
        float rbz = R[2][0] * bx + R[2][1] * by + R[2][2] * bz;
        float az = (A.pz + A.dpz) + rbz;
        float t = __fmul_rn(az, inv_uz);                  // rounded on its own (never fused)
        float l = t - kWheelR;
        const bool hit = uz > kUzMin && l < kRest;
        float x = kRest - fmaxf(l, 0.f);
        float wrz = A.wx * rby - A.wy * rbx;                // (w x rb).z
        float xdot = __fmul_rn(-(A.vz + wrz), inv_uz);
        // the damper engages over the first kDampRamp of compression:
        // the normal force is continuous at touchdown
        const float Ni = fmaxf(0.f, kKSusp * x + kCSusp * xdot * fminf(1.f, x / kDampRamp));
        N[i] = hit ? Ni : 0.f;
        rcx[i] = hit ? rbx - t * ux : 0.f;
        rcy[i] = hit ? rby - t * uy : 0.f;
        rcz[i] = hit ? rbz - t * uz : 0.f;
    }

    // 4. predicted velocities
    float Fx = fcx, Fy = fcy, Fz = -kMass * kG;
    float Tx = 0.f, Ty = 0.f, Tz = tcz - kLambdaYaw * A.wz;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        Fz += N[i];
        Tx += rcy[i] * N[i];
        Ty -= rcx[i] * N[i];
    }
    // angular momentum L = R I R^T w, through the body frame (each sum in one fixed
    // rounding order, so that every kernel inlining this step rounds it alike)
    auto dot3 = [](float a0, float b0, float a1, float b1, float a2, float b2) {
        return __fmaf_rn(a2, b2, __fmaf_rn(a1, b1, __fmul_rn(a0, b0)));
    };
    const float wbx = dot3(R[0][0], A.wx, R[1][0], A.wy, R[2][0], A.wz);
    const float wby = dot3(R[0][1], A.wx, R[1][1], A.wy, R[2][1], A.wz);
    const float wbz = dot3(R[0][2], A.wx, R[1][2], A.wy, R[2][2], A.wz);
    const float lbx = __fmul_rn(kIxx, wbx), lby = __fmul_rn(kIyy, wby), lbz = __fmul_rn(kIzz, wbz);
    float Lx = dot3(R[0][0], lbx, R[0][1], lby, R[0][2], lbz);
    float Ly = dot3(R[1][0], lbx, R[1][1], lby, R[1][2], lbz);
    float Lz = dot3(R[2][0], lbx, R[2][1], lby, R[2][2], lbz);
    float nx_ = Tx - (A.wy * Lz - A.wz * Ly);
    float ny_ = Ty - (A.wz * Lx - A.wx * Lz);
    float nz_ = Tz - (A.wx * Ly - A.wy * Lx);
    float v1x = A.vx + h * Fx * kInvMass, v1y = A.vy + h * Fy * kInvMass, v1z = A.vz + h * Fz * kInvMass;
    float w1x = A.wx + h * (Ii[0][0] * nx_ + Ii[0][1] * ny_ + Ii[0][2] * nz_);
    float w1y = A.wy + h * (Ii[1][0] * nx_ + Ii[1][1] * ny_ + Ii[1][2] * nz_);
    float w1z = A.wz + h * (Ii[2][0] * nx_ + Ii[2][1] * ny_ + Ii[2][2] * nz_);
    const float drive = h * thr * kTauDrive * kInvWheelI;
    float sp[4] = {A.s0 + drive, A.s1 + drive, A.s2, A.s3};

    // 5. friction impulses, friction circle per wheel; each wheel takes the
    // chassis share of one of four wheels (a Jacobi step relaxed by 1/4: no
    // overshoot, and continuous when a wheel unloads)
    const float ncf = 4.f;
    float sd, cd;
    sincosf(A.dl, &sd, &cd);
    float Px = 0.f, Py = 0.f, Lmx = 0.f, Lmy = 0.f, Lmz = 0.f;
    float sp2[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        // an unloaded wheel (or one whose forward direction has no planar part)
        // selects a zero impulse: the sums below then add +0, which changes no
        // sum that starts at +0, exactly as if the wheel were skipped
        const float c = i < 2 ? cd : 1.f, s = i < 2 ? sd : 0.f;
        float fwx = R[0][0] * c + R[0][1] * s;
        float fwy = R[1][0] * c + R[1][1] * s;
        const float fl2 = norm2(fwx, fwy);
        const bool ok = N[i] > 0.f && fl2 > 0.f;
        const float rfl = rsqrtf(fl2);
        float elx = __fmul_rn(fwx, rfl), ely = __fmul_rn(fwy, rfl);
        float etx = -ely, ety = elx;
        float vcx = v1x + (w1y * rcz[i] - w1z * rcy[i]);
        float vcy = v1y + (w1z * rcx[i] - w1x * rcz[i]);
        // r x e for e in the plane: (-rz ey, rz ex, rx ey - ry ex)
        float ax_ = -rcz[i] * ely, ay_ = rcz[i] * elx, az_ = rcx[i] * ely - rcy[i] * elx;
        float q1 = ax_ * (Ii[0][0] * ax_ + Ii[0][1] * ay_ + Ii[0][2] * az_) +
                   ay_ * (Ii[1][0] * ax_ + Ii[1][1] * ay_ + Ii[1][2] * az_) +
                   az_ * (Ii[2][0] * ax_ + Ii[2][1] * ay_ + Ii[2][2] * az_);
        float wl = kWheelR2OverI + ncf * (kInvMass + q1);
        float bx_ = -rcz[i] * ety, by_ = rcz[i] * etx, bz_ = rcx[i] * ety - rcy[i] * etx;
        float q2 = bx_ * (Ii[0][0] * bx_ + Ii[0][1] * by_ + Ii[0][2] * bz_) +
                   by_ * (Ii[1][0] * bx_ + Ii[1][1] * by_ + Ii[1][2] * bz_) +
                   bz_ * (Ii[2][0] * bx_ + Ii[2][1] * by_ + Ii[2][2] * bz_);
        float wt = ncf * (kInvMass + q2);
        float ul = sp[i] * kWheelR - (vcx * elx + vcy * ely);
        float ut = -(vcx * etx + vcy * ety);
        float jl = ul / wl, jt = ut / wt;
        float cap = A.mu * N[i] * h;
        const float j2 = norm2(jl, jt);
        float sc = j2 <= __fmul_rn(cap, cap) ? 1.f : __fmul_rn(cap, rsqrtf(j2));   // friction circle
        jl *= sc; jt *= sc;
        float Jx = ok ? jl * elx + jt * etx : 0.f, Jy = ok ? jl * ely + jt * ety : 0.f;
        Px += Jx; Py += Jy;
        Lmx += -rcz[i] * Jy;
        Lmy += rcz[i] * Jx;
        Lmz += rcx[i] * Jy - rcy[i] * Jx;
        sp2[i] = ok ? sp[i] - jl * kWheelR * kInvWheelI : sp[i];
    }
    const float bf = h * brk * kTauBrkF * kInvWheelI, br = h * brk * kTauBrkR * kInvWheelI;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float m = fmaxf(fabsf(sp2[i]) - (i < 2 ? bf : br), 0.f);
        sp2[i] = sp2[i] >= 0.f ? m : -m;
    }
    A.s0 = sp2[0]; A.s1 = sp2[1]; A.s2 = sp2[2]; A.s3 = sp2[3];

    // 6. apply impulses
    v1x += Px * kInvMass; v1y += Py * kInvMass;
    w1x += Ii[0][0] * Lmx + Ii[0][1] * Lmy + Ii[0][2] * Lmz;
    w1y += Ii[1][0] * Lmx + Ii[1][1] * Lmy + Ii[1][2] * Lmz;
    w1z += Ii[2][0] * Lmx + Ii[2][1] * Lmy + Ii[2][2] * Lmz;

    // 7. positions, attitude q += h/2 (0, w) (x) q, normalised
    A.dpx += h * v1x; A.dpy += h * v1y; A.dpz += h * v1z;
    float qw = A.qw, qx = A.qx, qy = A.qy, qz = A.qz;
    float dqw = -(w1x * qx + w1y * qy + w1z * qz);
    float dqx = w1x * qw + (w1y * qz - w1z * qy);
    float dqy = w1y * qw + (w1z * qx - w1x * qz);
    float dqz = w1z * qw + (w1x * qy - w1y * qx);
    qw += 0.5f * h * dqw; qx += 0.5f * h * dqx; qy += 0.5f * h * dqy; qz += 0.5f * h * dqz;
    const float rq = rsqrtf(__fmaf_rn(qz, qz, __fmaf_rn(qy, qy, __fmaf_rn(qx, qx, __fmul_rn(qw, qw)))));
    A.qw = __fmul_rn(qw, rq); A.qx = __fmul_rn(qx, rq); A.qy = __fmul_rn(qy, rq); A.qz = __fmul_rn(qz, rq);
    A.vx = v1x; A.vy = v1y; A.vz = v1z;
    A.wx = w1x; A.wy = w1y; A.wz = w1z;
}

// ------------------------------------------------------------------ road queries
struct Lane {
    int seg;
    float dist, lat, tx, ty;  // tangent oriented toward the goal, lat sign follows it
};

// swept three-circle TTC (App. D), clamped to [0, 10] s; behind or no root -> 10
__device__ __forceinline__ float ttc_pair(float pix, float piy, float hix, float hiy, float vix, float viy, float pjx,
                                          float pjy, float hjx, float hjy, float vjx, float vjy) {
    float bx, by;
    to_ego(hix, hiy, pjx - pix, pjy - piy, bx, by);
    if (bx < 0.f) return kTtcMax;
    float dvx = vjx - vix, dvy = vjy - viy;
    float A2 = dvx * dvx + dvy * dvy;
    {   // every circle centre is within kCircD of its car centre: if the centres never come
        // within 2 (r + d) of each other for t >= 0, no circle pair can touch
        const float px_ = pjx - pix, py_ = pjy - piy;
        const float pv = px_ * dvx + py_ * dvy;
        const float c2 = px_ * px_ + py_ * py_;
        const float dmin2 = (pv < 0.f && A2 > 0.f) ? c2 - pv * pv / A2 : c2;
        const float lim = 2.f * (kCircR + kCircD);
        if (dmin2 > lim * lim * (1.f + 1e-4f) + 1e-3f) return kTtcMax;
    }
    float best = kInf;
#pragma unroll
    for (int a = -1; a <= 1; ++a)
#pragma unroll
        for (int b = -1; b <= 1; ++b) {
            float dx = (pjx + (float)b * kCircD * hjx) - (pix + (float)a * kCircD * hix);
            float dy = (pjy + (float)b * kCircD * hjy) - (piy + (float)a * kCircD * hiy);
            float B = 2.f * (dx * dvx + dy * dvy);
            float C = dx * dx + dy * dy - 4.f * kCircR * kCircR;
            float t;
            if (C <= 0.f) t = 0.f;
            else if (B >= 0.f) continue;
            else {
                float disc = B * B - 4.f * A2 * C;
                if (disc < 0.f) continue;
                t = 2.f * C / (-B + sqrtf(disc));
            }
            best = fminf(best, t);
        }
    if (best == kInf) return kTtcMax;
    return clampf(best, 0.f, kTtcMax);
}

// DRAC (App. G reading): closing speed^2 / (2 gap), the gap measured along the
// line of centres between the two footprints' reaches
__device__ __forceinline__ float drac_pair(float pix, float piy, float hix, float hiy, float vix, float viy, float pjx,
                                           float pjy, float hjx, float hjy, float vjx, float vjy) {
    float rx = pjx - pix, ry = pjy - piy;
    float dist = sqrtf(rx * rx + ry * ry);
    if (!(dist > 0.f)) return 0.f;
    float ux = rx / dist, uy = ry / dist;
    float vr = -((vjx - vix) * ux + (vjy - viy) * uy);
    float ei = kHalfLen * fabsf(hix * ux + hiy * uy) + kHalfWid * fabsf(-hiy * ux + hix * uy);
    float ej = kHalfLen * fabsf(hjx * ux + hjy * uy) + kHalfWid * fabsf(-hjy * ux + hjx * uy);
    float gap = fmaxf(dist - ei - ej, kDracGapFloor);
    return vr > 0.f ? vr * vr / (2.f * gap) : 0.f;
}

__device__ __forceinline__ float penalty(float alpha, float tau, float pmax) {
    return fminf(alpha / fmaxf(tau, kTtcFloor), pmax);
}

// exchange area of one world: footprints, velocities, goals of its agents
constexpr int kMaxPairs = 64;   // candidate contact pairs of a warp handled pair-parallel per substep
struct Exch {
    float px[32], py[32], hx[32], hy[32], vx[32], vy[32], dx[32], dy[32], gx[32], gy[32];
    // one substep's candidate contact pairs (lo < hi): per lane the first pair id and the mask of its
    // partners above it; the pair list and each pair's force (fx, fy, tz)
    int poff[32];
    uint32_t pmask[32];
    int plist[kMaxPairs];
    float4 pf[kMaxPairs];
};

__device__ __forceinline__ void publish(Exch& E, int lane, const Agent& A, float hx, float hy) {
    E.px[lane] = A.px; E.py[lane] = A.py;
    E.hx[lane] = hx; E.hy[lane] = hy;
    E.vx[lane] = A.vx; E.vy[lane] = A.vy;
    E.dx[lane] = A.dpx; E.dy[lane] = A.dpy;
    E.gx[lane] = A.gx; E.gy[lane] = A.gy;
}

__device__ __forceinline__ void load_agent(const DevState& st, int a, Agent& A) {
    float4 p = st.pos[a], q = st.quat[a], v = st.vel[a], w = st.angv[a], s = st.spin[a], g = st.goal[a];
    A.px = p.x; A.py = p.y; A.pz = p.z; A.dl = p.w;
    A.qw = q.x; A.qx = q.y; A.qy = q.z; A.qz = q.w;
    A.vx = v.x; A.vy = v.y; A.vz = v.z; A.dd = v.w;
    A.wx = w.x; A.wy = w.y; A.wz = w.z; A.mu = w.w;
    A.s0 = s.x; A.s1 = s.y; A.s2 = s.z; A.s3 = s.w;
    A.gx = g.x; A.gy = g.y; A.sx = g.z; A.sy = g.w;
    A.peak = st.peak_drac[a];
    A.meta = st.meta[a];
    A.step = st.step[a];
    A.episode = st.episode[a];
    A.dpx = A.dpy = A.dpz = 0.f;
}

__device__ __forceinline__ void store_agent(const DevState& st, int a, const Agent& A) {
    st.pos[a] = make_float4(A.px, A.py, A.pz, A.dl);
    st.quat[a] = make_float4(A.qw, A.qx, A.qy, A.qz);
    st.vel[a] = make_float4(A.vx, A.vy, A.vz, A.dd);
    st.angv[a] = make_float4(A.wx, A.wy, A.wz, A.mu);
    st.spin[a] = make_float4(A.s0, A.s1, A.s2, A.s3);
    st.goal[a] = make_float4(A.gx, A.gy, A.sx, A.sy);
    st.peak_drac[a] = A.peak;
    st.meta[a] = A.meta;
    st.step[a] = A.step;
    st.episode[a] = A.episode;
}

__device__ __forceinline__ bool finite_agent(const Agent& A) {
    float s = A.px + A.py + A.pz + A.dl + A.qw + A.qx + A.qy + A.qz + A.vx + A.vy + A.vz + A.dd + A.wx + A.wy +
              A.wz + A.s0 + A.s1 + A.s2 + A.s3;
    return isfinite(s) && isfinite(A.px) && isfinite(A.vx);
}

__constant__ float c_mu_table[4][3] = {{0.90f, 0.85f, 0.60f},   // dry       (asphalt, concrete, gravel)
                                       {0.70f, 0.65f, 0.50f},   // light rain
                                       {0.50f, 0.45f, 0.40f},   // heavy rain
                                       {0.30f, 0.25f, 0.20f}};  // snow

// place agent at (x, y) heading psi with speed v0, static equilibrium, rolling wheels
// Static friction of the modified ALL weather-to-friction model (App. B) at
// 13.89 m/s: the printed mu_static(h) curve points of surface s (0 AC, 1 SMA,
// 2 OGFC) at h = 0, 0.1, ..., 0.8 mm joined linearly, then linearly down to the
// 1e-3 floor at the 0.85 mm aquaplaning threshold, the floor beyond; the film
// comes in hundredths of a millimetre.
__constant__ float c_all_mu[3][9] = {
    {1.1048f, 1.0657f, 1.0161f, 0.9593f, 0.9039f, 0.8595f, 0.8302f, 0.8134f, 0.8044f},   // AC
    {1.2043f, 1.1618f, 1.1078f, 1.0461f, 0.9857f, 0.9374f, 0.9056f, 0.8874f, 0.8776f},   // SMA
    {1.3368f, 1.2898f, 1.2301f, 1.1617f, 1.0948f, 1.0413f, 1.0061f, 0.9860f, 0.9753f}};  // OGFC
constexpr float kAllFloor = 1e-3f;
constexpr uint32_t kAllCutCmm = 85;
__device__ __forceinline__ float all_mu_static(uint32_t s, uint32_t film_cmm) {
    const float* m = c_all_mu[s > 2 ? 2 : s];
    if (film_cmm >= kAllCutCmm) return kAllFloor;
    if (film_cmm >= 80u) return m[8] + (kAllFloor - m[8]) * ((float)(film_cmm - 80u) / (float)(kAllCutCmm - 80u));
    const uint32_t k = film_cmm / 10u, r = film_cmm % 10u;
    return m[k] + (m[k + 1] - m[k]) * ((float)r / 10.f);
}
// the weather token's first entry: precip / 3 (table model) or h / h_norm, h_norm = 1 mm (Eq. weather_obs)
__device__ __forceinline__ float weather_level(uint32_t wb, bool all_model) {
    return all_model ? (float)wb * 0.01f : (float)wb / 3.f;
}

__device__ __forceinline__ void place_agent(Agent& A, float x, float y, float psi, float v0, float gx, float gy,
                                            bool all_model) {
    float s, c, sh, ch;
    sincosf(psi, &s, &c);
    sincosf(0.5f * psi, &sh, &ch);
    A.px = x; A.py = y; A.pz = kZStar; A.dl = 0.f;
    A.qw = ch; A.qx = 0.f; A.qy = 0.f; A.qz = sh;
    A.vx = v0 * c; A.vy = v0 * s; A.vz = 0.f; A.dd = 0.f;
    A.wx = A.wy = A.wz = 0.f;
    float om = v0 / kWheelR;
    A.s0 = A.s1 = A.s2 = A.s3 = om;
    A.gx = gx; A.gy = gy; A.sx = x; A.sy = y;
    uint32_t pc = A.meta & 0xFFu, sc = (A.meta >> 8) & 0xFFu;
    A.mu = all_model ? all_mu_static(sc, pc) : c_mu_table[pc > 3 ? 3 : pc][sc > 2 ? 2 : sc];
    A.peak = 0.f;
    A.step = 0;
    A.meta = with_status(A.meta, kAlive);
}

__device__ __forceinline__ void park_agent(Agent& A) {
    A.px = kParkX; A.py = 0.f;
    A.vx = A.vy = A.vz = 0.f;
    A.wx = A.wy = A.wz = 0.f;
    A.s0 = A.s1 = A.s2 = A.s3 = 0.f;
    A.meta = with_status(A.meta, kParked);
}

// spawn candidate r of agent a (handle index; its draws use its index in the
// whole CSR, rd.agent_base + a) for episode ep (App. J reading)
// a world without lane points spawns its slot k at (0, k * spacing), heading +x
// (cslot: the candidate's index in rd.cands, -1 for the fallback)
__device__ void spawn_candidate(const DevRoads& rd, int w, int a, int slot, int ep, int r, unsigned long long seed,
                                float& x, float& y, float& psi, float& gx, float& gy, float& v0, int& cslot) {
    const int2 cw = __ldg(&rd.cand[w]);
    x = 0.f; y = (float)slot * kSpawnSpacing; psi = 0.f; gx = kSpawnGoalMin; gy = y;
    cslot = -1;
    if (cw.y > 0) {
        uint32_t pick = (uint32_t)(reset_draw(seed, rd.agent_base + a, ep, r, 0) >> 32) % (uint32_t)cw.y;
        cslot = cw.x + (int)pick;
        int k = __ldg(&rd.cands[cslot]);
        float4 p = __ldg(&rd.pt[k]);
        x = p.x; y = p.y;
        psi = atan2f(p.w, p.z);
        float dg = kSpawnGoalMin + (kSpawnGoalMax - kSpawnGoalMin) * u24(reset_draw(seed, rd.agent_base + a, ep, r, 1));
        // the first point j after k with arc(k, j) >= dg (the polyline's last point
        // if none): binary search over the cumulative arc lengths
        const int k1 = __ldg(&rd.pend[k]);
        const float ak = __ldg(&rd.arc[k]);
        int lo = k + 1, hi = k1;                      // answer in [lo, hi], hi = none
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(&rd.arc[mid]) - ak >= dg) hi = mid; else lo = mid + 1;
        }
        const int g = lo < k1 ? lo : k1 - 1;
        float4 G = __ldg(&rd.pt[g]);
        gx = G.x; gy = G.y;
    }
    v0 = kSpawnVMin + (kSpawnVMax - kSpawnVMin) * u24(reset_draw(seed, rd.agent_base + a, ep, r, 2));
}


// ------------------------------------------------------------------ warp-cooperative road queries
// Keys order candidates lexicographically by (squared distance, index): the
// float bits of a non-negative d^2 are monotone as an unsigned integer.
constexpr unsigned long long kKeyInf = ~0ull;

__device__ __forceinline__ unsigned long long key_of(float d2, int idx) {
    return ((unsigned long long)__float_as_uint(d2) << 32) | (unsigned)idx;
}
__device__ __forceinline__ float key_d2(unsigned long long k) { return __uint_as_float((unsigned)(k >> 32)); }
__device__ __forceinline__ int key_idx(unsigned long long k) { return k == kKeyInf ? -1 : (int)(unsigned)k; }
__device__ __forceinline__ unsigned long long umin64(unsigned long long a, unsigned long long b) { return a < b ? a : b; }
__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) { return a < b ? b : a; }
__device__ __forceinline__ unsigned long long shfl64(unsigned long long v, int src) {
    unsigned lo = __shfl_sync(kFull, (unsigned)v, src), hi = __shfl_sync(kFull, (unsigned)(v >> 32), src);
    return ((unsigned long long)hi << 32) | lo;
}
__device__ __forceinline__ unsigned long long shfl_xor64(unsigned long long v, int m) {
    unsigned lo = __shfl_xor_sync(kFull, (unsigned)v, m), hi = __shfl_xor_sync(kFull, (unsigned)(v >> 32), m);
    return ((unsigned long long)hi << 32) | lo;
}
// the warp's smallest 64-bit value: the smallest high word, then the smallest
// low word among the lanes holding it (two warp reductions)
__device__ __forceinline__ unsigned long long warp_min64(unsigned long long v) {
    const unsigned hi = __reduce_min_sync(kFull, (unsigned)(v >> 32));
    const unsigned lo = __reduce_min_sync(kFull, (unsigned)(v >> 32) == hi ? (unsigned)v : 0xFFFFFFFFu);
    return ((unsigned long long)hi << 32) | lo;
}
// bitonic sort of one key per lane, ascending with the lane index
__device__ __forceinline__ unsigned long long warp_sort32(unsigned long long v, int lane) {
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            unsigned long long o = shfl_xor64(v, j);
            const bool asc = (lane & k) == 0, lo = (lane & j) == 0;
            v = (lo == asc) ? umin64(v, o) : umax64(v, o);
        }
    return v;
}
// merge a sorted running top-32 with 32 new (unsorted) candidates; returns the 32 smallest, sorted
__device__ __forceinline__ unsigned long long merge32(unsigned long long run, unsigned long long cand, int lane) {
    cand = warp_sort32(cand, lane);
    unsigned long long m = umin64(run, shfl64(cand, 31 - lane));   // bitonic, holds the 32 smallest
#pragma unroll
    for (int j = 16; j > 0; j >>= 1) {
        unsigned long long o = shfl_xor64(m, j);
        m = (lane & j) == 0 ? umin64(m, o) : umax64(m, o);
    }
    return m;
}

// The smallest 32 of the unique keys buf[0, cnt), cnt <= 64, by rank: a key's
// rank is the number of held keys below it, and the keys of rank < 32 are
// written back to buf at their rank, so buf[0, min(cnt, 32)) ends ascending.
// Every lane ranks its (at most two) keys against all of them (broadcast
// reads, no shuffles).  Returns min(cnt, 32).
__device__ __forceinline__ int rank_keep32(unsigned long long* buf, int cnt, int lane) {
    const unsigned long long k0 = lane < cnt ? buf[lane] : kKeyInf;
    const unsigned long long k1 = lane + 32 < cnt ? buf[lane + 32] : kKeyInf;
    int r0 = 0, r1 = 0;
#pragma unroll 4
    for (int i = 0; i < cnt; ++i) {
        const unsigned long long k = buf[i];
        r0 += k < k0 ? 1 : 0;
        r1 += k < k1 ? 1 : 0;
    }
    __syncwarp();
    if (lane < cnt && r0 < 32) buf[r0] = k0;
    if (lane + 32 < cnt && r1 < 32) buf[r1] = k1;
    __syncwarp();
    return cnt < 32 ? cnt : 32;
}

// One world's road blob as the queries see it: in shared memory when the
// block staged it, else in global memory (generic pointers either way).
struct WRoads {
    const uint16_t* coff;   // [nx*ny + 1] cell offsets into the sorted records
    const float4* seg;      // sorted segment records (x, y, x', y')
    const uint32_t* info;   // local input index | type << 16 | kInfo* bits
    const float4* edge;     // edge segments (a, b), sorted by edge-grid cell
    const uint16_t* eoff;   // [ex*ey + 1] edge-grid cell offsets into edge
    float x0, y0, inv_c, inv_ce;
    int nx, ny, ecnt, q0, ex, ey;
};

__device__ __forceinline__ WRoads view_of(const DevGrid& g, const unsigned char* base) {
    WRoads v;
    v.coff = reinterpret_cast<const uint16_t*>(base);
    v.seg = reinterpret_cast<const float4*>(base + g.o_seg);
    v.info = reinterpret_cast<const uint32_t*>(base + g.o_info);
    v.edge = reinterpret_cast<const float4*>(base + g.o_edge);
    v.eoff = reinterpret_cast<const uint16_t*>(base + g.o_eoff);
    v.x0 = g.x0; v.y0 = g.y0; v.inv_c = g.inv_c; v.inv_ce = g.inv_ce;
    v.nx = g.nx; v.ny = g.ny; v.ecnt = g.ecnt; v.q0 = g.q0; v.ex = g.ex; v.ey = g.ey;
    return v;
}

// Starting radius of a query from last step's answer d measured at h: the
// distance to the k-th nearest object grows by at most |p - h| (triangle
// inequality), so d + |p - h| (padded for rounding) already holds the previous
// answer's objects.  Unknown (d = 0) or far hints give the default r0.  The
// queries stay exact whatever the radius: they grow it until it is enough.
__device__ __forceinline__ float hint_radius(const float* hnt, int which, float px, float py, float r0) {
    const float d = hnt[which];
    const float dx = px - hnt[2], dy = py - hnt[3];
    const float jump = sqrtf(norm2(dx, dy));
    if (!(d > 0.f) || !(jump < kHintJump)) return r0;
    return d + jump * 1.0001f + 1e-3f;
}

// keys of road candidates: (d^2 bits, local input index, sorted position);
// the order is (d^2, input index), the position only locates the record
__device__ __forceinline__ unsigned long long rkey(float d2, uint32_t info, int pos) {
    return key_of(d2, (int)(((info & 0xFFFFu) << 16) | (uint32_t)pos));
}
__device__ __forceinline__ int rkey_pos(unsigned long long k) { return (int)(k & 0xFFFFull); }
__device__ __forceinline__ int rkey_local(unsigned long long k) { return (int)((k >> 16) & 0xFFFFull); }

// Grid rows covering the square [q - R, q + R]^2: every point outside it is
// at least R away from q.  `all` when the square covers the whole grid.
struct Rows {
    int cx0, cx1, cy0, cy1;
    bool all;
};
__device__ __forceinline__ Rows rows_covering(const WRoads& g, float qx, float qy, float R) {
    const float fx0 = fminf(fmaxf((qx - R - g.x0) * g.inv_c, -1.f), (float)g.nx);
    const float fx1 = fminf(fmaxf((qx + R - g.x0) * g.inv_c, -1.f), (float)g.nx);
    const float fy0 = fminf(fmaxf((qy - R - g.y0) * g.inv_c, -1.f), (float)g.ny);
    const float fy1 = fminf(fmaxf((qy + R - g.y0) * g.inv_c, -1.f), (float)g.ny);
    Rows w;
    w.cx0 = max((int)floorf(fx0), 0); w.cx1 = min((int)floorf(fx1), g.nx - 1);
    w.cy0 = max((int)floorf(fy0), 0); w.cy1 = min((int)floorf(fy1), g.ny - 1);
    w.all = w.cx0 == 0 && w.cy0 == 0 && w.cx1 == g.nx - 1 && w.cy1 == g.ny - 1;
    return w;
}

// The records of the cells in columns cx0..cx1 of rows cy0..cy1, in batches of
// 32 (lane t takes one record of each batch): the rows' bounds are read in one
// step (one row per lane, up to 32 rows at a time) and their ranges flattened
// by a prefix sum, so a batch can span rows, and the next batch's loads are
// issued before `body` runs on the current one.  body(sg, m, i, has) is called
// by every lane, `has` false past the last record; the queries built on it
// keep the order-independent answers (a minimum, a set of smallest keys, an
// any), so the batching does not change them.
template <class F>
__device__ __forceinline__ void scan_cells(const WRoads& v, const Rows& w, int lane, F&& body) {
    if (w.cx0 > w.cx1) return;
    for (int r0 = w.cy0; r0 <= w.cy1; r0 += 32) {
        int s = 0, n = 0;
        if (r0 + lane <= w.cy1) {
            const int row = (r0 + lane) * v.nx;
            s = v.coff[row + w.cx0];
            n = v.coff[row + w.cx1 + 1] - s;
        }
        int incl = n;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        const int total = __shfl_sync(kFull, incl, 31);
        const int shift = s - (incl - n);          // record index of flattened j in this row: j + shift
        // record index of flattened candidate j: its row is the number of rows
        // whose inclusive end is <= j (incl is non-decreasing over the lanes)
        auto locate = [&](int j) {
            int r = 0;
#pragma unroll
            for (int st = 16; st > 0; st >>= 1)
                if (__shfl_sync(kFull, incl, r + st - 1) <= j) r += st;
            return j + __shfl_sync(kFull, shift, r);
        };
        int i = locate(lane);
        bool has = lane < total;
        float4 sg = make_float4(0.f, 0.f, 0.f, 0.f);
        uint32_t m = 0u;
        if (has) { sg = v.seg[i]; m = v.info[i]; }
        for (int base = 0; base < total; base += 32) {
            const int jn = base + 32 + lane;
            const int in = locate(jn);
            const bool hn = jn < total;
            float4 sgn = make_float4(0.f, 0.f, 0.f, 0.f);
            uint32_t mn = 0u;
            if (hn) { sgn = v.seg[in]; mn = v.info[in]; }
            body(sg, m, i, has);
            sg = sgn; m = mn; i = in; has = hn;
        }
    }
}

// the warp's smallest key, and in r the record of the lane that held it (keys
// are unique: they carry the record's position)
__device__ __forceinline__ unsigned long long warp_min_rec(unsigned long long k, float4& r) {
    const unsigned long long m = warp_min64(k);
    const unsigned win = __ballot_sync(kFull, k == m);
    const int src = win ? __ffs(win) - 1 : 0;
    r.x = __shfl_sync(kFull, r.x, src); r.y = __shfl_sync(kFull, r.y, src);
    r.z = __shfl_sync(kFull, r.z, src); r.w = __shfl_sync(kFull, r.w, src);
    return m;
}

// tangent, lateral offset and distance of the nearest lane segment from its
// key and its record r = (a, b), before the orientation toward the goal
__device__ __forceinline__ Lane lane_raw_of(const WRoads& v, unsigned long long best, const float4& r, float qx,
                                            float qy) {
    Lane L;
    if (best == kKeyInf) { L.seg = -1; L.dist = kInf; L.lat = 0.f; L.tx = L.ty = 0.f; return L; }
    L.seg = v.q0 + rkey_local(best);
    const float ex = r.z - r.x, ey = r.w - r.y;
    const float nn = sqrtf(norm2(ex, ey));
    L.tx = ex / nn; L.ty = ey / nn;
    L.lat = cross2(L.tx, L.ty, qx - r.x, qy - r.y);
    L.dist = sqrtf(key_d2(best));
    return L;
}
// the tangent oriented toward the goal g (App. G), the lateral offset's sign following it
__device__ __forceinline__ void lane_orient(Lane& L, float qx, float qy, float gx, float gy) {
    if (L.seg >= 0 && dot2(L.tx, gx - qx, L.ty, gy - qy) < 0.f) { L.tx = -L.tx; L.ty = -L.ty; L.lat = -L.lat; }
}
__device__ __forceinline__ Lane lane_of(const WRoads& v, unsigned long long best, const float4& r, float qx, float qy,
                                        float gx, float gy) {
    Lane L = lane_raw_of(v, best, r, qx, qy);
    lane_orient(L, qx, qy, gx, gy);
    return L;
}

// lane-forbidden test of one edge segment against the footprint's three
// circles, given d0 = its squared distance from the centre circle's centre q:
// the side circles (kCircD from q) can only touch a segment closer to q than
// kCircD + the touch distance, tested first (a conservative bound)
constexpr float kForbLim = (kCircR + kEdgeHalfWidth) * (kCircR + kEdgeHalfWidth);
constexpr float kForbSide = (kCircD + kCircR + kEdgeHalfWidth) * (kCircD + kCircR + kEdgeHalfWidth) * 1.0001f + 1e-4f;
__device__ __forceinline__ bool forb_touch(const float4& sg, float d0, float qx, float qy, float hx, float hy) {
    if (d0 < kForbLim) return true;
    if (!(d0 < kForbSide)) return false;
    bool f = false;
#pragma unroll
    for (int c = -1; c <= 1; c += 2) {
        const float cx_ = qx + (float)c * kCircD * hx, cy_ = qy + (float)c * kCircD * hy;
        if (seg_dist2(sg.x, sg.y, sg.z, sg.w, cx_, cy_) < kForbLim) f = true;
    }
    return f;
}

// nearest driving-lane segment (App. G), exact: a segment within D of q starts
// inside the square of half-size D + 3 m around q (no segment is longer than
// 3 m), so scanning the cells of the square of half-size S finds every lane
// segment within S - 3; S grows until one is found.  On the first pass the
// same scan runs the lane-forbidden test of the footprint's three circles
// against the road-edge segments (App. G) when `forb` is given: the square
// then also covers every edge segment that can touch a circle.
__device__ Lane coop_nearest_lane_raw(const WRoads& v, float qx, float qy, float R, int lane, bool* forb = nullptr,
                                      float hx = 1.f, float hy = 0.f) {
    float S = R + kSegReach;
    if (forb) S = fmaxf(S, kCircD + kCircR + kEdgeHalfWidth + kSegReach);
    bool edges = forb != nullptr, f = false;
    unsigned long long best = kKeyInf;
    float4 brec = make_float4(0.f, 0.f, 0.f, 0.f);
    for (;;) {
        const Rows w = rows_covering(v, qx, qy, S);
        const float Rl = S - kSegReach;
        const float lim = w.all ? kInf : Rl * Rl * (1.f - 1e-5f);
        best = kKeyInf;
        const uint32_t want = kInfoLane | (edges ? kInfoEdge : 0u);
        scan_cells(v, w, lane, [&](const float4& sg, uint32_t m, int i, bool has) {
            if (!has || !(m & kInfoSegNext) || !(m & want)) return;
            const float d0 = seg_dist2(sg.x, sg.y, sg.z, sg.w, qx, qy);
            if (m & kInfoLane) {
                const unsigned long long k = rkey(d0, m, i);
                if (d0 < lim && k < best) { best = k; brec = sg; }
            } else if (forb_touch(sg, d0, qx, qy, hx, hy)) {
                f = true;
            }
        });
        best = warp_min_rec(best, brec);
        if (edges) { *forb = __any_sync(kFull, f); edges = false; }
        if (best != kKeyInf || w.all) break;
        S = Rl * kGrow + kSegReach;
    }
    return lane_raw_of(v, best, brec, qx, qy);
}
__device__ __forceinline__ Lane coop_nearest_lane(const WRoads& v, float qx, float qy, float gx, float gy, float R,
                                                  int lane, bool* forb = nullptr, float hx = 1.f, float hy = 0.f) {
    Lane L = coop_nearest_lane_raw(v, qx, qy, R, lane, forb, hx, hy);
    lane_orient(L, qx, qy, gx, gy);
    return L;
}

// Candidate keys (kKeyInf: none) of a batch are appended to the warp's buffer
// (64 keys); whenever more than 32 are held, the 32 smallest are kept, and the
// largest of them tightens the admission threshold (a key at or above it can
// no longer be among the 32 nearest).  `sorted` tells whether buf[0, cnt) is
// the ascending result of a trim with nothing appended since.
__device__ __forceinline__ void collect_keys(unsigned long long key, int lane, unsigned lt, unsigned long long* buf,
                                             int& cnt, unsigned long long& thr, bool& sorted) {
    const unsigned mk = __ballot_sync(kFull, key != kKeyInf);
    if (!mk) return;
    if (key != kKeyInf) buf[cnt + __popc(mk & lt)] = key;
    cnt += __popc(mk);
    sorted = false;
    __syncwarp();
    if (cnt > 32) {
        cnt = rank_keep32(buf, cnt, lane);
        thr = umin64(thr, buf[31]);
        sorted = true;
    }
}
// lane t's key of the t-th smallest held key (kKeyInf past cnt); buf sorted first if needed
__device__ __forceinline__ unsigned long long held_key(unsigned long long* buf, int& cnt, bool sorted, int lane) {
    if (!sorted) cnt = rank_keep32(buf, cnt, lane);
    const unsigned long long k = lane < cnt ? buf[lane] : kKeyInf;
    __syncwarp();
    return k;
}

// The running selection of the 32 smallest candidate keys of one warp, in one
// of two forms with the same result (the 32 smallest, ascending, lane t
// holding the t-th): RANK keeps them in the warp's buffer and ranks them
// (fewer dependent steps: for blocks whose warps wait on one another), else
// every 32 collected are merged bitonically into a running top-32 in
// registers (fewer instructions: for grids of independent warps that fill the
// issue slots).
template <bool RANK>
struct Sel32 {
    unsigned long long* buf;
    unsigned lt;
    int lane, cnt;
    bool sorted;
    unsigned long long run;
    __device__ __forceinline__ Sel32(unsigned long long* b, int l)
        : buf(b), lt((1u << l) - 1u), lane(l), cnt(0), sorted(true), run(kKeyInf) {}
    __device__ __forceinline__ void add(unsigned long long key, unsigned long long& thr) {
        if constexpr (RANK) {
            collect_keys(key, lane, lt, buf, cnt, thr, sorted);
        } else {
            const unsigned mk = __ballot_sync(kFull, key != kKeyInf);
            if (key != kKeyInf) buf[cnt + __popc(mk & lt)] = key;
            cnt += __popc(mk);
            __syncwarp();
            if (cnt >= 32) {
                run = merge32(run, buf[lane], lane);
                const unsigned long long rest = lane < cnt - 32 ? buf[32 + lane] : kKeyInf;
                __syncwarp();
                if (lane < cnt - 32) buf[lane] = rest;
                cnt -= 32;
                thr = umin64(thr, shfl64(run, 31));
                __syncwarp();
            }
        }
    }
    // lane t's key of the t-th smallest; full: 32 were found
    __device__ __forceinline__ unsigned long long result(bool& full) {
        if constexpr (RANK) {
            const unsigned long long k = held_key(buf, cnt, sorted, lane);
            full = cnt == 32;
            return k;
        } else {
            if (cnt > 0) run = merge32(run, lane < cnt ? buf[lane] : kKeyInf, lane);
            __syncwarp();
            full = shfl64(run, 31) != kKeyInf;
            return run;
        }
    }
};

// the 32 nearest road points (all types), exact; lane t returns the t-th key.
// Only points closer than R compete; if fewer than 32 are, R grows.
// buf: 64 keys of shared memory owned by the calling warp.
template <bool RANK>
__device__ unsigned long long coop_knn32(const WRoads& v, float qx, float qy, float R, int lane,
                                         unsigned long long* buf) {
    for (;;) {
        const Rows w = rows_covering(v, qx, qy, R);
        unsigned long long thr = w.all ? kKeyInf : key_of(R * R * (1.f - 1e-5f), 0);
        Sel32<RANK> sel(buf, lane);
        scan_cells(v, w, lane, [&](const float4& P, uint32_t m, int i, bool has) {
            unsigned long long key = kKeyInf;
            if (has) {
                const float dx = P.x - qx, dy = P.y - qy;
                key = rkey(norm2(dx, dy), m, i);
                if (key >= thr) key = kKeyInf;
            }
            sel.add(key, thr);
        });
        bool full;
        const unsigned long long run = sel.result(full);
        if (full || w.all) return run;
        R *= kGrow;
    }
}

// One pass over the cells around q for the three point queries of an agent
// at once: the 32 nearest road points (radius R32), the nearest driving-lane
// segment (radius Rl) and the lane-forbidden test of the footprint's circles.
// The scanned square covers all three; each answer is exact when its own
// radius held enough candidates, else that query is redone alone with a
// growing radius (coop_knn32 / coop_nearest_lane).  Returns the lane; lane t
// of the warp gets the t-th nearest point's key in *key.
template <bool RANK>
__device__ Lane coop_point_queries(const WRoads& v, float qx, float qy, float gx, float gy, float hx, float hy,
                                   float R32, float Rl, int lane, unsigned long long* buf, bool* forb,
                                   unsigned long long* key) {
    const float S = fmaxf(fmaxf(Rl + kSegReach, kCircD + kCircR + kEdgeHalfWidth + kSegReach), R32);
    const Rows w = rows_covering(v, qx, qy, S);
    const float Rle = S - kSegReach;                  // every lane segment within Rle is seen
    const float lim_l = w.all ? kInf : Rle * Rle * (1.f - 1e-5f);
    unsigned long long thr = w.all ? kKeyInf : key_of(R32 * R32 * (1.f - 1e-5f), 0);
    unsigned long long best = kKeyInf;
    float4 brec = make_float4(0.f, 0.f, 0.f, 0.f);
    bool f = false;
    Sel32<RANK> sel(buf, lane);
    scan_cells(v, w, lane, [&](const float4& sg, uint32_t m, int i, bool has) {
        unsigned long long k = kKeyInf;
        if (has) {
            const float dx = sg.x - qx, dy = sg.y - qy;
            k = rkey(norm2(dx, dy), m, i);
            if (k >= thr) k = kKeyInf;
            if ((m & kInfoSegNext) && (m & (kInfoLane | kInfoEdge))) {
                const float d0 = seg_dist2(sg.x, sg.y, sg.z, sg.w, qx, qy);
                if (m & kInfoLane) {
                    const unsigned long long kl = rkey(d0, m, i);
                    if (d0 < lim_l && kl < best) { best = kl; brec = sg; }
                } else if (forb_touch(sg, d0, qx, qy, hx, hy)) {
                    f = true;
                }
            }
        }
        sel.add(k, thr);
    });
    bool full;
    const unsigned long long run = sel.result(full);
    *forb = __any_sync(kFull, f);
    best = warp_min_rec(best, brec);
    // too few points within R32: the 32 nearest alone, from a larger radius
    *key = (full || w.all) ? run : coop_knn32<RANK>(v, qx, qy, R32 * kGrow, lane, buf);
    if (best == kKeyInf && !w.all)                   // no lane within Rle: the nearest lane alone
        return coop_nearest_lane(v, qx, qy, gx, gy, Rle * kGrow, lane);
    return lane_of(v, best, brec, qx, qy, gx, gy);
}

// time for the constant-velocity ray from an agent to reach the nearest road
// edge segment within 40 m (App. G).  GRID: scan only the edge-grid cells the
// ray can reach; else every edge of the world, four loads per lane in flight
// (fewer registers and round trips: the split step's query kernel).  Both give
// the same answer: the earliest accepted hit, and the edges GRID skips cannot
// be hit.
template <bool GRID>
__device__ float coop_edge_ray(const WRoads& v, float px, float py, float vx, float vy, int lane) {
    // ray p + v t against the edge segments; the acceptance tests t >= 0,
    // 0 <= s <= 1 and |v| t <= 40 m are evaluated multiplied through by the
    // denominator (sign-aware), and only accepted hits divide.  A segment whose
    // start is farther than 40 m + 3 m cannot be hit within the horizon.
    const float speed = sqrtf(vx * vx + vy * vy);
    if (!(speed > 0.f)) return kInf;   // a ray that does not move hits nothing (every denominator is 0)
    const float reach2 = (kEdgeHorizon + kSegReach) * (kEdgeHorizon + kSegReach);
    float t_best = kInf;
    auto hit = [&](const float4& sg4) {
        const float apx = sg4.x - px, apy = sg4.y - py;
        if (norm2(apx, apy) > reach2) return;
        const float exx = sg4.z - sg4.x, eyy = sg4.w - sg4.y;
        const float den = cross2(vx, vy, exx, eyy);
        if (den == 0.f) return;
        const float nt = cross2(apx, apy, exx, eyy), ns = cross2(apx, apy, vx, vy);
        const bool ok = den > 0.f ? (nt >= 0.f && ns >= 0.f && ns <= den && speed * nt <= kEdgeHorizon * den)
                                  : (nt <= 0.f && ns <= 0.f && ns >= den && speed * nt >= kEdgeHorizon * den);
        if (ok) t_best = fminf(t_best, __fadd_rn(nt / den, 0.f));   // >= 0 (+0 for a zero time)
    };
    if (!GRID) {
        constexpr int kU = 4;
        for (int i0 = lane; i0 < v.ecnt; i0 += 32 * kU) {
            float4 e[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u)
                if (i0 + 32 * u < v.ecnt) e[u] = v.edge[i0 + 32 * u];
#pragma unroll
            for (int u = 0; u < kU; ++u)
                if (i0 + 32 * u < v.ecnt) hit(e[u]);
        }
        return __uint_as_float(__reduce_min_sync(kFull, __float_as_uint(t_best)));
    }
    // an accepted hit lies on the ray within 40 m and on a segment no longer than
    // 3 m, so the segment's start lies in the ray segment's bounding box grown by
    // 3 m; 1 m more covers rounding.  Only the edge-grid cells of that box are scanned.
    const float ux = vx / speed * kEdgeHorizon, uy = vy / speed * kEdgeHorizon, pad = kSegReach + 1.f;
    const float bx0 = fminf(px, px + ux) - pad, bx1 = fmaxf(px, px + ux) + pad;
    const float by0 = fminf(py, py + uy) - pad, by1 = fmaxf(py, py + uy) + pad;
    const int cx0 = max((int)floorf(fminf(fmaxf((bx0 - v.x0) * v.inv_ce, -1.f), (float)v.ex)), 0);
    const int cx1 = min((int)floorf(fminf(fmaxf((bx1 - v.x0) * v.inv_ce, -1.f), (float)v.ex)), v.ex - 1);
    const int cy0 = max((int)floorf(fminf(fmaxf((by0 - v.y0) * v.inv_ce, -1.f), (float)v.ey)), 0);
    const int cy1 = min((int)floorf(fminf(fmaxf((by1 - v.y0) * v.inv_ce, -1.f), (float)v.ey)), v.ey - 1);
    if (cx0 <= cx1)
        for (int cy = cy0; cy <= cy1; ++cy) {   // a row's cells are one contiguous range of edges
            const int e0 = v.eoff[cy * v.ex + cx0], e1 = v.eoff[cy * v.ex + cx1 + 1];
            constexpr int kU = 2;               // two segments per lane in flight
            for (int i0 = e0 + lane; i0 < e1; i0 += 32 * kU) {
                float4 e[kU];
#pragma unroll
                for (int u = 0; u < kU; ++u)
                    if (i0 + 32 * u < e1) e[u] = v.edge[i0 + 32 * u];
#pragma unroll
                for (int u = 0; u < kU; ++u)
                    if (i0 + 32 * u < e1) hit(e[u]);
            }
        }
    // times are >= +0 or +inf, ordered like their bit patterns
    return __uint_as_float(__reduce_min_sync(kFull, __float_as_uint(t_best)));
}

// road-point features of the observation (App. D analogue) from a k-NN key
// and the point's record (r, m)
__device__ __forceinline__ void point_features_of(const float4& r, uint32_t m, float ehx, float ehy, float epx,
                                                  float epy, float f[kObsPt]) {
    // road direction at the point: toward the next point of the polyline,
    // from the previous one at a polyline's end
    float ddx = r.z - r.x, ddy = r.w - r.y;
    if (!(m & kInfoHasNext)) { ddx = -ddx; ddy = -ddy; }
    const float nn = sqrtf(norm2(ddx, ddy));
    if (nn > 0.f) { ddx /= nn; ddy /= nn; } else { ddx = ddy = 0.f; }
    float bx, by, dbx, dby;
    to_ego(ehx, ehy, r.x - epx, r.y - epy, bx, by);
    to_ego(ehx, ehy, ddx, ddy, dbx, dby);
    f[0] = bx / 10.f; f[1] = by / 10.f; f[2] = dbx; f[3] = dby;
    f[4] = (float)((m >> 16) & 0xFFu) / 20.f;
    f[5] = (m & kInfoEdge) ? 1.f : 0.f;
    f[6] = 1.f;
}
__device__ __forceinline__ void point_features(const WRoads& v, unsigned long long key, float ehx, float ehy,
                                               float epx, float epy, float f[kObsPt]) {
    const int pos = rkey_pos(key);
    point_features_of(v.seg[pos], v.info[pos], ehx, ehy, epx, epy, f);
}

// ------------------------------------------------------------------ dynamics surrogate
// Heading frame at t: rotation by psi about z (psi of the body x axis).
// Features (30): z, tilt quaternion q_psi^-1 q (4), v and w in the heading
// frame (3 + 3), wheel spins (4), suspension compressions and rates (4 + 4),
// steer angle and rate, decoded action (3), mu, 0.
// Targets (16): R_psi^T dp - v_h dt (3), body rotation vector of q_t^-1 q_t+1
// - w_body dt (3), R_psi^T v_t+1 - v_h (3), R_psi^T w_t+1 - w_h (3), dOmega (4).
constexpr float kSurrMuMin = 0.3f, kSurrVMax = 35.0f, kSurrCosTilt = 0.98480775f;   // cos 10 deg
constexpr float kSurrReach = 4.8466483f + 2.0f;   // two circumradii of the footprint + 2 m

struct Frame {
    float c, s;      // cos, sin of psi
};
__device__ __forceinline__ Frame frame_of(float qw, float qx, float qy, float qz) {
    float hx, hy;
    heading_of(qw, qx, qy, qz, hx, hy);
    Frame f;
    f.c = hx; f.s = hy;
    return f;
}
__device__ __forceinline__ void to_h(const Frame& f, float x, float y, float& hx_, float& hy_) {
    hx_ = f.c * x + f.s * y;
    hy_ = -f.s * x + f.c * y;
}
__device__ __forceinline__ void from_h(const Frame& f, float x, float y, float& wx, float& wy) {
    wx = f.c * x - f.s * y;
    wy = f.s * x + f.c * y;
}

__device__ void surr_features(const Agent& A, float thr, float dstar, float brk, float* x) {
    const Frame f = frame_of(A.qw, A.qx, A.qy, A.qz);
    const float psi = atan2f(f.s, f.c);
    float sh, ch;
    sincosf(0.5f * psi, &sh, &ch);
    x[0] = A.pz;
    x[1] = ch * A.qw + sh * A.qz;
    x[2] = ch * A.qx + sh * A.qy;
    x[3] = ch * A.qy - sh * A.qx;
    x[4] = ch * A.qz - sh * A.qw;
    to_h(f, A.vx, A.vy, x[5], x[6]);
    x[7] = A.vz;
    to_h(f, A.wx, A.wy, x[8], x[9]);
    x[10] = A.wz;
    x[11] = A.s0; x[12] = A.s1; x[13] = A.s2; x[14] = A.s3;
    float R[3][3];
    quat_to_mat(A.qw, A.qx, A.qy, A.qz, R);
    const float uz = R[2][2];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float bx = i < 2 ? kHardX : -kHardX, by = (i & 1) == 0 ? kHardY : -kHardY, bz = kHardZ;
        const float rbx = R[0][0] * bx + R[0][1] * by + R[0][2] * bz;
        const float rby = R[1][0] * bx + R[1][1] * by + R[1][2] * bz;
        const float rbz = R[2][0] * bx + R[2][1] * by + R[2][2] * bz;
        float xc = 0.f, xd = 0.f;
        if (uz > kUzMin) {
            const float t = (A.pz + rbz) / uz, l = t - kWheelR;
            if (l < kRest) {
                xc = kRest - fmaxf(l, 0.f);
                xd = -(A.vz + (A.wx * rby - A.wy * rbx)) / uz;
            }
        }
        x[15 + i] = xc;
        x[19 + i] = xd;
    }
    x[23] = A.dl; x[24] = A.dd;
    x[25] = thr; x[26] = dstar; x[27] = brk;
    x[28] = A.mu;
    x[29] = 0.f;
}

// rotation vector of a unit quaternion (shortest rotation)
__device__ __forceinline__ void quat_log(float w, float x, float y, float z, float& rx, float& ry, float& rz) {
    if (w < 0.f) { w = -w; x = -x; y = -y; z = -z; }
    const float n = sqrtf(x * x + y * y + z * z);
    const float ang = 2.f * atan2f(n, w);
    const float k = n > 1e-12f ? ang / n : 2.f;
    rx = k * x; ry = k * y; rz = k * z;
}

// targets of one step from the start state (p0, q0, v0, w0, s0) and the end state A
__device__ void surr_targets(float4 p0, float4 q0, float4 v0, float4 w0, float4 s0, const Agent& A, float dt,
                             float* y) {
    const Frame f = frame_of(q0.x, q0.y, q0.z, q0.w);
    float dph_x, dph_y, vh0x, vh0y, vh1x, vh1y, wh0x, wh0y, wh1x, wh1y;
    to_h(f, A.px - p0.x, A.py - p0.y, dph_x, dph_y);
    to_h(f, v0.x, v0.y, vh0x, vh0y);
    to_h(f, A.vx, A.vy, vh1x, vh1y);
    to_h(f, w0.x, w0.y, wh0x, wh0y);
    to_h(f, A.wx, A.wy, wh1x, wh1y);
    y[0] = dph_x - vh0x * dt;
    y[1] = dph_y - vh0y * dt;
    y[2] = (A.pz - p0.z) - v0.z * dt;
    // q_rel = q0^-1 q1 (body frame at t)
    const float aw = q0.x, ax = -q0.y, ay = -q0.z, az = -q0.w;
    const float rw = aw * A.qw - ax * A.qx - ay * A.qy - az * A.qz;
    const float rx = aw * A.qx + ax * A.qw + (ay * A.qz - az * A.qy);
    const float ry = aw * A.qy + ay * A.qw + (az * A.qx - ax * A.qz);
    const float rz = aw * A.qz + az * A.qw + (ax * A.qy - ay * A.qx);
    float tx, ty, tz;
    quat_log(rw, rx, ry, rz, tx, ty, tz);
    float R[3][3];
    quat_to_mat(q0.x, q0.y, q0.z, q0.w, R);
    const float wbx = R[0][0] * w0.x + R[1][0] * w0.y + R[2][0] * w0.z;   // R^T w
    const float wby = R[0][1] * w0.x + R[1][1] * w0.y + R[2][1] * w0.z;
    const float wbz = R[0][2] * w0.x + R[1][2] * w0.y + R[2][2] * w0.z;
    y[3] = tx - wbx * dt; y[4] = ty - wby * dt; y[5] = tz - wbz * dt;
    y[6] = vh1x - vh0x; y[7] = vh1y - vh0y; y[8] = A.vz - v0.z;
    y[9] = wh1x - wh0x; y[10] = wh1y - wh0y; y[11] = A.wz - w0.z;
    y[12] = A.s0 - s0.x; y[13] = A.s1 - s0.y; y[14] = A.s2 - s0.z; y[15] = A.s3 - s0.w;
}

// apply denormalised targets d[16] to the start state (p0 ... s0): the chassis part of A
__device__ void surr_apply(float4 p0, float4 q0, float4 v0, float4 w0, float4 s0, const float* d, float dt, Agent& A) {
    const Frame f = frame_of(q0.x, q0.y, q0.z, q0.w);
    float vh0x, vh0y, wh0x, wh0y, ox, oy;
    to_h(f, v0.x, v0.y, vh0x, vh0y);
    to_h(f, w0.x, w0.y, wh0x, wh0y);
    from_h(f, d[0] + vh0x * dt, d[1] + vh0y * dt, ox, oy);
    A.px = p0.x + ox; A.py = p0.y + oy; A.pz = p0.z + (d[2] + v0.z * dt);
    float R[3][3];
    quat_to_mat(q0.x, q0.y, q0.z, q0.w, R);
    const float tx = d[3] + (R[0][0] * w0.x + R[1][0] * w0.y + R[2][0] * w0.z) * dt;
    const float ty = d[4] + (R[0][1] * w0.x + R[1][1] * w0.y + R[2][1] * w0.z) * dt;
    const float tz = d[5] + (R[0][2] * w0.x + R[1][2] * w0.y + R[2][2] * w0.z) * dt;
    const float ang = sqrtf(tx * tx + ty * ty + tz * tz);
    float sa, ca;
    sincosf(0.5f * ang, &sa, &ca);
    const float k = ang > 1e-12f ? sa / ang : 0.5f;
    const float ew = ca, ex = k * tx, ey = k * ty, ez = k * tz;   // exp of the rotation vector
    float qw = q0.x * ew - q0.y * ex - q0.z * ey - q0.w * ez;       // q0 (x) e
    float qx = q0.x * ex + q0.y * ew + (q0.z * ez - q0.w * ey);
    float qy = q0.x * ey + q0.z * ew + (q0.w * ex - q0.y * ez);
    float qz = q0.x * ez + q0.w * ew + (q0.y * ey - q0.z * ex);
    const float qn = sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
    A.qw = qw / qn; A.qx = qx / qn; A.qy = qy / qn; A.qz = qz / qn;
    from_h(f, vh0x + d[6], vh0y + d[7], A.vx, A.vy);
    A.vz = v0.z + d[8];
    from_h(f, wh0x + d[9], wh0y + d[10], A.wx, A.wy);
    A.wz = w0.z + d[11];
    A.s0 = s0.x + d[12]; A.s1 = s0.y + d[13]; A.s2 = s0.z + d[14]; A.s3 = s0.w + d[15];
}

// gate of lane `lane` given the exchange area at the start of the step
__device__ __forceinline__ bool surr_gate(const Exch& E, int base, int n, int lane, uint32_t alive_bits,
                                          const Agent& A, float dt) {
    if (!((alive_bits >> lane) & 1u)) return false;
    if (A.mu < kSurrMuMin) return false;
    if (A.vx * A.vx + A.vy * A.vy + A.vz * A.vz > kSurrVMax * kSurrVMax) return false;
    if (1.f - 2.f * (A.qx * A.qx + A.qy * A.qy) < kSurrCosTilt) return false;
    for (int j = base; j < base + n; ++j) {
        if (j == lane || !((alive_bits >> j) & 1u)) continue;
        const float dvx = E.vx[j] - A.vx, dvy = E.vy[j] - A.vy;
        const float reach = kSurrReach + sqrtf(dvx * dvx + dvy * dvy) * dt;
        const float dx = E.px[j] - A.px, dy = E.py[j] - A.py;
        if (norm2(dx, dy) <= reach * reach) return false;
    }
    return true;
}

// per-agent results of the cooperative queries

}  // namespace

// ------------------------------------------------------------------ road staging
// A block copies the road blobs of its pack's worlds into shared memory with
// one bulk (TMA) copy per world, completing on an mbarrier; the copy is issued
// before the physics and waited for before the first road query.  Every wait
// is bounded (1 s): on expiry the error word gets bit 1 and the queries read
// the blobs from global memory instead.
constexpr uint64_t kStageWaitNs = 1000000000ull;
constexpr uint32_t kStageSpinMax = 1u << 30;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ bool stage_done(uint64_t* bar) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(bar))
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t now_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
// bounded wait for the staging copy: false when it has not landed within limit_ns
__device__ bool stage_wait(uint64_t* bar, uint64_t limit_ns) {
    if (stage_done(bar)) return true;
    const uint64_t t0 = now_ns();
    for (uint32_t i = 0; i < kStageSpinMax; ++i) {
        if (stage_done(bar)) return true;
        if ((i & 63) == 63 && now_ns() - t0 > limit_ns) break;
    }
    return false;
}
// warp 0: lane 0 arms the barrier for `total` bytes, lane t copies world t;
// with `withhold` the barrier is only initialised (nothing will complete it)
__device__ void stage_issue(const unsigned char* gblob, const DevGrid* sg, const int* woff, int nworlds, int total,
                            unsigned char* dst, uint64_t* bar, int lane, bool withhold) {
    if (lane == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (!withhold)
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(total)
                         : "memory");
    }
    __syncwarp();
    if (!withhold && lane < nworlds && sg[lane].bytes > 0)
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         smem_addr(dst + woff[lane])),
                     "l"(gblob + sg[lane].blob), "r"(sg[lane].bytes), "r"(smem_addr(bar))
                     : "memory");
}

// ====================================================================== step building blocks
// Used by the fused world kernel and by the split step alike (the same inline
// code, so that both give bit-identical results).

// a lane of the agent warp: its slot in the block's pack and its world
struct Slot {
    bool has;       // the lane holds an agent
    int a;          // agent index (the pack's first agent for lanes without one)
    int wl, w;      // pack-local world, world id
    int base, n;    // the world's first slot and its agent count
};

__device__ __forceinline__ Slot slot_of(const int4& pk, const int* s_slot_w, const int* s_wbase, const int* s_wn,
                                        int lane, bool warp0) {
    Slot c;
    c.has = warp0 && lane < pk.w;
    c.a = pk.z + (c.has ? lane : 0);
    c.wl = 0; c.w = pk.x; c.base = 0; c.n = 0;
    if (c.has) {
        c.wl = s_slot_w[lane];
        c.w = pk.x + c.wl;
        c.base = s_wbase[c.wl];
        c.n = s_wn[c.wl];
    }
    return c;
}

// the pack's slot tables (warp 0, lanes < worlds of the pack)
__device__ __forceinline__ void pack_tables(const WorldArgs& args, const int4& pk, int lane, int* s_slot_w,
                                            int* s_wbase, int* s_wn) {
    if (lane < pk.y) {
        const int4 wd = __ldg(&args.rd.world[pk.x + lane]);
        s_wbase[lane] = wd.x - pk.z;
        s_wn[lane] = wd.y;
        for (int k = 0; k < wd.y; ++k) s_slot_w[wd.x - pk.z + k] = lane;
    }
    __syncwarp();
}

// physics of one control step for the lanes of the agent warp (Sec. 4.1,
// App. F): action decode, substeps with footprint contact through the
// exchange area every substep, the surrogate for gated agents, the
// non-finite check; the post-step pose is published in E at the end
// One control step of the kinematic bicycle (Sec. 4.4 ablation backend): the
// front wheel steers delta = 30 deg x steer, the speed follows the rectified
// throttle / brake accelerations and never reverses, and with the centre of
// mass midway between the axles the slip angle is beta = atan(tan(delta) / 2):
//   v' = max(0, |v| + a dt), p' = p + v' (cos, sin)(psi + beta) dt,
//   psi' = psi + v' sin(beta) / (WB / 2) dt.
// The chassis stays level at the static ride height; no suspension, contact
// response or lateral slip.
__device__ __forceinline__ void bicycle_step(Agent& A, const float* act, float dt) {
    const float thr = clampf(act[0], 0.f, 1.f), brk = clampf(act[2], 0.f, 1.f);
    const float delta = kBikeThetaMax * clampf(act[1], -1.f, 1.f);
    const float beta = atanf(0.5f * tanf(delta));
    const float psi = 2.f * atan2f(A.qz, A.qw);
    const float v = sqrtf(A.vx * A.vx + A.vy * A.vy);
    const float v1 = fmaxf(0.f, v + (kBikeADrive * thr - kBikeABrake * brk) * dt);
    const float r = v1 / (0.5f * kWheelbase) * sinf(beta);
    A.px += v1 * cosf(psi + beta) * dt;
    A.py += v1 * sinf(psi + beta) * dt;
    const float psi1 = psi + r * dt;
    A.pz = kZStar;
    A.qw = cosf(0.5f * psi1); A.qx = 0.f; A.qy = 0.f; A.qz = sinf(0.5f * psi1);
    A.vx = v1 * cosf(psi1 + beta); A.vy = v1 * sinf(psi1 + beta); A.vz = 0.f;
    A.wx = 0.f; A.wy = 0.f; A.wz = r;
    A.s0 = A.s1 = A.s2 = A.s3 = v1 / kWheelR;
    A.dl = delta; A.dd = 0.f;
}

// the physics a step kernel is compiled with: the raycast vehicle, the vehicle
// with the learned surrogate's gate, or the kinematic bicycle (the variants not
// launched stay out of the kernel's code)
enum PhysKind { kPhysVehicle = 0, kPhysSurrogate = 1, kPhysBicycle = 2 };
__host__ __device__ inline int phys_of(const WorldArgs& a) {
    return a.dynamics == 1 ? kPhysBicycle : (a.surr_mode != 0 ? kPhysSurrogate : kPhysVehicle);
}

// contact culling (lanes_physics): the distance an agent may move in a control
// step, and whether slot j is a contact candidate of slot i (i's view: the
// sums in this order, so that every kernel evaluating it rounds alike)
__device__ __forceinline__ float cull_budget(float vx, float vy, float T) {
    return __fmaf_rn(sqrtf(norm2(vx, vy)), T, 1.f);
}
__device__ __forceinline__ bool cull_near(float pxi, float pyi, float bi, float pxj, float pyj, float bj) {
    const float reach = kPairCullR + bi + bj + 0.01f;
    return norm2(pxj - pxi, pyj - pyi) <= __fmul_rn(reach, reach);
}

// every slot's contact candidates (the s = 0 set of lanes_physics), one slot
// per warp at a time over warps w0, w0 + nwarps, ...; lane l holds slot l's
// start-of-step position and budget
__device__ __forceinline__ void pairs_near(const int4& pk, const int* s_slot_w, const int* s_wbase, const int* s_wn,
                                           int w0, int nwarps, int lane, float px, float py, float budget,
                                           unsigned* s_near) {
    for (int i = w0; i < pk.w; i += nwarps) {
        const float bi = __shfl_sync(kFull, budget, i);
        const float pxi = __shfl_sync(kFull, px, i), pyi = __shfl_sync(kFull, py, i);
        const int wl = s_slot_w[i];
        const int base = s_wbase[wl], n = s_wn[wl];
        const bool hit = lane >= base && lane < base + n && lane != i && cull_near(pxi, pyi, bi, px, py, budget);
        const unsigned mask = __ballot_sync(kFull, hit);
        if (lane == 0) s_near[i] = mask;
    }
}

template <int PHYS>
// act: the lane's raw actions (throttle, steer, brake), loaded by the caller
// pre_near: every slot's contact candidates, written by other warps of the
// block, which arrive on named barrier 2 (bar_threads threads with this warp)
// when they are; nullptr: this warp computes them
__device__ __forceinline__ void lanes_physics(const WorldArgs& args, const Slot& c, int lane, Agent& A, bool& alive,
                                              bool& nonfin, float& prevx, float& prevy, float& hx, float& hy,
                                              Exch& E, float3 act, const unsigned* pre_near = nullptr,
                                              int bar_threads = 0) {
    const DevState& st = args.st;
    const int a = c.a, base = c.base, n = c.n;
    float thr = 0.f, dstar = 0.f, brk = 0.f;
    if (alive) {
        thr = clampf(act.x, 0.f, 1.f);
        dstar = kThetaMax * clampf(act.y, -1.f, 1.f);
        brk = clampf(act.z, 0.f, 1.f);
    }
    prevx = A.px; prevy = A.py;
    bool gated = false;
    if (PHYS == kPhysBicycle) {   // the bicycle backend replaces the substeps (no contact response)
        const float av[3] = {act.x, act.y, act.z};
        if (alive) bicycle_step(A, av, args.h * args.substeps);
        if (alive && !finite_agent(A)) {
            nonfin = true;
            park_agent(A);
            alive = false;
            atomicOr(args.out.error_word, 1u);
        }
        heading_of(A.qw, A.qx, A.qy, A.qz, hx, hy);
        publish(E, lane, A, hx, hy);
        __syncwarp();
        return;
    }
    // contact candidates: the pairs of the world that can come within the cull
    // distance during this control step.  Lane i may move |v_i| T + 1 m (its
    // budget) before the set is rebuilt, so a pair farther apart at the start
    // than the cull distance + both budgets is culled at every substep, and
    // skipping it is exact (a culled pair adds +0, and a force sum that starts
    // at +0 is never -0).  A lane that exceeds its budget rebuilds the set as
    // all pairs of its world for the remaining substeps.
    const float T = args.h * args.substeps;
    const float budget = cull_budget(A.vx, A.vy, T);
    uint32_t near = 0u;
    if (pre_near) {
        named_bar_sync(2, bar_threads);
        near = c.has ? pre_near[lane] : 0u;
    }
    bool wide = false;
    for (int s = 0; s < args.substeps; ++s) {
        float sx_, sy_;
        heading_of(A.qw, A.qx, A.qy, A.qz, sx_, sy_);
        publish(E, lane, A, sx_, sy_);
        const uint32_t alive_bits = __ballot_sync(kFull, alive);
        __syncwarp();
        if (PHYS == kPhysSurrogate && s == 0 && args.surr_mode != 0)
            gated = surr_gate(E, base, n, lane, alive_bits, A, args.h * args.substeps);
        if (s == 0 && !pre_near) {
            // every slot of the pack in turn (a warp-uniform count), its position and
            // budget by shuffles
            const int jend = __reduce_max_sync(kFull, (uint32_t)(base + n));
#pragma unroll 4
            for (int j = 0; j < jend; ++j) {
                const float bj = __shfl_sync(kFull, budget, j);
                const float pxj = __shfl_sync(kFull, A.px, j), pyj = __shfl_sync(kFull, A.py, j);
                if (j >= base && j < base + n && j != lane && cull_near(A.px, A.py, budget, pxj, pyj, bj))
                    near |= 1u << j;
            }
        }
        if (!wide && __any_sync(kFull, alive && A.dpx * A.dpx + A.dpy * A.dpy > budget * budget)) wide = true;
        const uint32_t cand = (wide ? 0xFFFFFFFFu : near) & alive_bits;
        float fcx = 0.f, fcy = 0.f, tcz = 0.f;
        // candidate pairs (lo < hi) of the world, compacted over the warp: each pair's force is
        // computed once, by one lane, then every lane sums its partners in ascending order (the
        // order, and so the rounding, of a per-lane loop over its partners)
        const uint32_t wmask = (n >= 32 ? 0xFFFFFFFFu : ((1u << n) - 1u)) << base;
        const uint32_t above = lane < 31 ? (0xFFFFFFFFu << (lane + 1)) : 0u;
        const uint32_t mine = alive ? (cand & above & wmask) : 0u;
        // candidate sets are symmetric: with no lane holding a partner above it there
        // is no pair, and the forces stay +0 (the body step below is the only one,
        // so its rounding is the same whichever way a substep goes)
        if (__any_sync(kFull, mine != 0u)) {
            // exclusive prefix sum of the pair counts (at most 31, five bits) over the
            // lanes: one ballot per bit, all independent
            const int pc = __popc(mine);
            const uint32_t lt = (1u << lane) - 1u;
            int poff = 0, npairs = 0;
#pragma unroll
            for (int b = 0; b < 5; ++b) {
                const uint32_t bb = __ballot_sync(kFull, (pc >> b) & 1);
                poff += __popc(bb & lt) << b;
                npairs += __popc(bb) << b;
            }
            if (npairs <= kMaxPairs) {
                E.poff[lane] = poff;
                E.pmask[lane] = mine;
                for (uint32_t mm = mine, k = (uint32_t)poff; mm; mm &= mm - 1u, ++k) E.plist[k] = (lane << 8) | (__ffs(mm) - 1);
                __syncwarp();
                for (int p = lane; p < npairs; p += 32) {
                    const int lo = E.plist[p] >> 8, hi = E.plist[p] & 0xFF;
                    float fx, fy, tz;
                    pair_force(E.px[lo], E.py[lo], E.dx[lo], E.dy[lo], E.hx[lo], E.hy[lo], E.vx[lo], E.vy[lo],
                               E.px[hi], E.py[hi], E.dx[hi], E.dy[hi], E.hx[hi], E.hy[hi], E.vx[hi], E.vy[hi],
                               fx, fy, tz);
                    E.pf[p] = make_float4(fx, fy, tz, 0.f);
                }
                __syncwarp();
                if (alive) {
                    for (uint32_t pm = cand & wmask & ~(1u << lane); pm; pm &= pm - 1u) {   // ascending j
                        const int j = __ffs(pm) - 1;
                        const int lo = min(lane, j), hi = max(lane, j);
                        const float4 f = E.pf[E.poff[lo] + __popc(E.pmask[lo] & ((1u << hi) - 1u))];
                        if (lane == lo) { fcx -= f.x; fcy -= f.y; } else { fcx += f.x; fcy += f.y; }
                        tcz += f.z;
                    }
                }
            } else if (alive) {   // many candidates (all pairs of a crowded world): a loop per lane
                for (uint32_t pm = cand & wmask & ~(1u << lane); pm; pm &= pm - 1u) {   // ascending j
                    const int j = __ffs(pm) - 1;
                    const int lo = min(lane, j), hi = max(lane, j);
                    float fx, fy, tz;
                    pair_force(E.px[lo], E.py[lo], E.dx[lo], E.dy[lo], E.hx[lo], E.hy[lo], E.vx[lo], E.vy[lo],
                               E.px[hi], E.py[hi], E.dx[hi], E.dy[hi], E.hx[hi], E.hy[hi], E.vx[hi], E.vy[hi],
                               fx, fy, tz);
                    if (lane == lo) { fcx -= fx; fcy -= fy; } else { fcx += fx; fcy += fy; }
                    tcz += tz;
                }
            }
        }
        __syncwarp();
        if (alive) {
            if (gated && args.surr_mode == 1) steer_substep(A, dstar, args.h);   // chassis from the surrogate
            else body_substep(A, thr, dstar, brk, fcx, fcy, tcz, args.h);
        }
    }
    A.px += A.dpx; A.py += A.dpy; A.pz += A.dpz;
    A.dpx = A.dpy = A.dpz = 0.f;
    if (gated) {
        // the start-of-step state is still in global memory (stored after the physics)
        const float4 p0 = st.pos[a], q0 = st.quat[a], v0 = st.vel[a], w0 = st.angv[a], s0 = st.spin[a];
        float d[kSurrOut];
        const float* yn = args.surr_y + (size_t)a * kSurrOut;
#pragma unroll
        for (int k = 0; k < kSurrOut; ++k) d[k] = args.surr_stats[k] + args.surr_stats[kSurrOut + k] * yn[k];
        const float dt = args.h * args.substeps;
        if (args.surr_mode == 1) {
            surr_apply(p0, q0, v0, w0, s0, d, dt, A);
            atomicAdd(args.surr_count, 1u);
        } else {
            Agent P = A;
            surr_apply(p0, q0, v0, w0, s0, d, dt, P);
            const float ex = P.px - A.px, ey = P.py - A.py, ez = P.pz - A.pz;
            atomicMax(args.audit_err, __float_as_uint(sqrtf(ex * ex + ey * ey + ez * ez)));
        }
    }
    if (alive && !finite_agent(A)) {
        nonfin = true;
        park_agent(A);
        alive = false;
        atomicOr(args.out.error_word, 1u);
    }
    heading_of(A.qw, A.qx, A.qy, A.qz, hx, hy);
    publish(E, lane, A, hx, hy);
}

// road-point block of one agent's observation (all lanes of a warp).  With
// `need` (the agent was respawned, or every agent is observed afresh) the
// nearest lane is first recomputed from radius rlane into *L; the 32 nearest points start from the hinted
// radius (the default after a respawn); the hints are updated.  orow gets the
// 32 x 7 features (zeros when !alive), knn_row (may be null) the indices.
// A respawned agent sits on a lane point, so its lane query starts from
// kSpawnLaneR (the query still grows its radius until the answer is exact).
constexpr float kSpawnLaneR = 1.0f;

template <bool RANK>
__device__ __forceinline__ void agent_road_block(const WRoads& v, bool alive, bool need, float px, float py,
                                                 float gx, float gy, float hx, float hy, float* hnt, int lane,
                                                 unsigned long long* kbuf, float* orow, int32_t* knn_row, Lane* L,
                                                 float rlane = kLaneR0) {
    unsigned long long key = kKeyInf;
    if (alive) {
        if (need) {
            *L = coop_nearest_lane(v, px, py, gx, gy, rlane, lane);
            __syncwarp();
            if (lane == 0) hnt[1] = L->seg >= 0 ? L->dist : 0.f;
        }
        const float r32 = need ? kKnnR0 : hint_radius(hnt, 0, px, py, kKnnR0);
        __syncwarp();
        key = coop_knn32<RANK>(v, px, py, r32, lane, kbuf);
        const unsigned long long last = shfl64(key, 31);
        if (lane == 0) {
            hnt[0] = last != kKeyInf ? sqrtf(key_d2(last)) : 0.f;
            hnt[2] = px;
            hnt[3] = py;
        }
    }
    float f[kObsPt] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (key != kKeyInf) point_features(v, key, hx, hy, px, py, f);
#pragma unroll
    for (int k = 0; k < kObsPt; ++k) orow[kObsPt * lane + k] = f[k];
    if (knn_row) knn_row[lane] = key != kKeyInf ? v.q0 + rkey_local(key) : -1;
}

// The road queries of one alive agent at its end-of-physics pose (all lanes of
// a warp), in one pass over the cells around it: the nearest lane with the
// lane-forbidden test (events) and the 32 nearest road points (the
// observation's road-point block, written to orow, indices to knn_row), then
// the edge ray; hv holds the agent's hints, which are updated through hnt.
// Returns the events' answers (every lane).
template <bool RANK>
__device__ __forceinline__ AgentQ agent_step_queries(const WRoads& v, float px, float py, float gx, float gy, float hx,
                                                     float hy, float vx, float vy, const float (&hv)[4], float* hnt,
                                                     int lane, unsigned long long* kbuf, float* orow,
                                                     int32_t* knn_row) {
    bool forb = false;
    unsigned long long key = kKeyInf;
    const Lane L = coop_point_queries<RANK>(v, px, py, gx, gy, hx, hy, hint_radius(hv, 0, px, py, kKnnR0),
                                      hint_radius(hv, 1, px, py, kLaneR0), lane, kbuf, &forb, &key);
    // the observation's point records are fetched while the edge ray runs
    float4 prec = make_float4(0.f, 0.f, 0.f, 0.f);
    uint32_t pm = 0u;
    if (key != kKeyInf) { prec = v.seg[rkey_pos(key)]; pm = v.info[rkey_pos(key)]; }
    // the fused kernel (RANK) takes the edge grid; the split query kernel the linear scan
    const float tedge = coop_edge_ray<RANK>(v, px, py, vx, vy, lane);
    const unsigned long long last = shfl64(key, 31);
    __syncwarp();
    AgentQ q;
    q.seg = L.seg; q.dist = L.dist; q.lat = L.lat; q.tx = L.tx; q.ty = L.ty;
    q.tedge = tedge; q.forb = forb ? 1 : 0; q.need = 0;
    if (lane == 0) {
        hnt[0] = last != kKeyInf ? sqrtf(key_d2(last)) : 0.f;
        hnt[1] = L.seg >= 0 ? L.dist : 0.f;
        hnt[2] = px;
        hnt[3] = py;
    }
    float f[kObsPt] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (key != kKeyInf) point_features_of(prec, pm, hx, hy, px, py, f);
#pragma unroll
    for (int k = 0; k < kObsPt; ++k) orow[kObsPt * lane + k] = f[k];
    if (knn_row) knn_row[lane] = key != kKeyInf ? v.q0 + rkey_local(key) : -1;
    return q;
}

// Road-point block and nearest lane (into *L) of an agent standing exactly on
// the spawn candidate whose spawn-table entry is e (all lanes of a warp): the
// table holds the answers of the exact queries at that point, so the result
// equals agent_road_block's there bit for bit; the hints are updated as it
// would update them.
__device__ __forceinline__ void spawn_road_block(const SpawnQ* e, const WRoads& v, float px, float py, float gx,
                                                 float gy, float hx, float hy, float* hnt, int lane, float* orow,
                                                 int32_t* knn_row, Lane* L) {
    const int pos = e->pos[lane];
    Lane l;
    l.seg = e->seg; l.dist = e->dist; l.lat = e->lat; l.tx = e->tx; l.ty = e->ty;
    lane_orient(l, px, py, gx, gy);
    *L = l;
    if (lane == 0) {
        hnt[0] = e->d32;
        hnt[1] = l.seg >= 0 ? l.dist : 0.f;
        hnt[2] = px;
        hnt[3] = py;
    }
    float f[kObsPt] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    uint32_t m = 0u;
    if (pos != 0xFFFF) {
        m = v.info[pos];
        point_features_of(v.seg[pos], m, hx, hy, px, py, f);
    }
#pragma unroll
    for (int k = 0; k < kObsPt; ++k) orow[kObsPt * lane + k] = f[k];
    if (knn_row) knn_row[lane] = pos != 0xFFFF ? v.q0 + (int)(m & 0xFFFFu) : -1;
}

// Neighbour tables of a block: the 8 nearest agents of every slot and, per
// (slot, neighbour) pair, TTC and DRAC; the pairs are spread over every warp.
struct Nbr {
    int8_t nb[32][kK];
    float tt[32][kK], dr[32][kK];
    float hx[32], hy[32];     // heading of each slot for the observation (after respawns)
};

// The K nearest alive agents of every alive slot in `todo` (lexicographic
// (d^2, index) order, the order of knn_agents) and, with coll, the footprint
// overlaps of the collision event (App. G: SAT of the slot's footprint against
// every alive partner within the cull distance): one (slot, partner) pair per
// thread.  Phase 1 writes the squared distances into D[slot][partner] (inf for
// no partner) and sets bit i of *coll on an overlap; phase 2 counts each
// partner's rank among its slot's partners and writes the partners of rank < K
// to N.nb (every neighbour of a todo slot is written, -1 past the partners).
// Positions and headings come from the exchange area.
__device__ __forceinline__ void pairs_knn(const Exch& E, Nbr& N, float (*D)[32], const int* s_slot_w,
                                          const int* s_wbase, const int* s_wn, int m, uint32_t alive_bits,
                                          uint32_t todo, unsigned* coll, int tid, int nthreads) {
    for (int p = tid; p < m * 32; p += nthreads) {
        const int i = p >> 5, jj = p & 31;
        if (!((todo >> i) & 1u)) continue;
        if (jj < kK) N.nb[i][jj] = -1;
        const int wl = s_slot_w[i], base = s_wbase[wl], n = s_wn[wl];
        if (jj >= n) continue;
        const int j = base + jj;
        float d2 = kInf;
        if (j != i && ((alive_bits >> i) & 1u) && ((alive_bits >> j) & 1u)) {
            d2 = norm2(E.px[j] - E.px[i], E.py[j] - E.py[i]);
            if (coll && d2 <= kPairCull2) {
                float nx, ny;
                if (sat2d(E.px[i], E.py[i], E.hx[i], E.hy[i], E.px[j], E.py[j], E.hx[j], E.hy[j], nx, ny) > 0.f)
                    atomicOr(coll, 1u << i);
            }
        }
        D[i][jj] = d2;
    }
    __syncthreads();
    for (int p = tid; p < m * 32; p += nthreads) {
        const int i = p >> 5, jj = p & 31;
        if (!((todo >> i) & 1u)) continue;
        const int wl = s_slot_w[i], n = s_wn[wl];
        if (jj >= n) continue;
        const float dj = D[i][jj];
        if (!(dj < kInf)) continue;
        int rank = 0;
        for (int kk = 0; kk < n; ++kk) {
            const float dk = D[i][kk];
            rank += (dk < dj || (dk == dj && kk < jj)) ? 1 : 0;
        }
        if (rank < kK) N.nb[i][rank] = (int8_t)(s_wbase[wl] + jj);
    }
}

// K nearest alive other agents (lexicographic (d^2, index) order); local lane ids
// over the slots [base, base + n) of the lane's own world
__device__ __forceinline__ void knn_agents(const Exch& E, int base, int n, int lane, uint32_t alive_bits, float px,
                                           float py, int nb[kK]) {
    float key[kK];
#pragma unroll
    for (int t = 0; t < kK; ++t) { key[t] = kInf; nb[t] = -1; }
    for (int j = base; j < base + n; ++j) {
        if (j == lane || !((alive_bits >> j) & 1u)) continue;
        const float d2 = norm2(E.px[j] - px, E.py[j] - py);
        if (!(d2 < key[kK - 1])) continue;
        float ck = d2;
        int ci = j;
        bool ins = false;
#pragma unroll
        for (int t = 0; t < kK; ++t) {
            if (ins || ck < key[t]) {
                float tk = key[t]; key[t] = ck; ck = tk;
                int ti = nb[t]; nb[t] = ci; ci = ti;
                ins = true;
            }
        }
    }
}


// The same answers as pairs_knn for a block of one warp, a lane per slot:
// the lane's K nearest alive agents into N.nb[lane], and whether its footprint
// overlaps an alive agent's (the same squared distances and SAT tests, so the
// same results bit for bit)
__device__ __forceinline__ bool lanes_knn(const Exch& E, int base, int n, int lane, uint32_t alive_bits, bool alive,
                                          bool coll, Nbr& N) {
    int nb[kK];
    bool collided = false;
    knn_agents(E, base, n, lane, alive_bits, E.px[lane], E.py[lane], nb);
    if (!alive) {
#pragma unroll
        for (int t = 0; t < kK; ++t) nb[t] = -1;
    }
    if (coll && alive) {
        for (int j = base; j < base + n && !collided; ++j) {
            if (j == lane || !((alive_bits >> j) & 1u)) continue;
            if (norm2(E.px[j] - E.px[lane], E.py[j] - E.py[lane]) > kPairCull2) continue;
            float nx, ny;
            if (sat2d(E.px[lane], E.py[lane], E.hx[lane], E.hy[lane], E.px[j], E.py[j], E.hx[j], E.hy[j], nx, ny) > 0.f)
                collided = true;
        }
    }
#pragma unroll
    for (int t = 0; t < kK; ++t) N.nb[lane][t] = (int8_t)nb[t];
    return collided;
}

// events and rewards (App. G), first part, lanes of the agent warp: lane terms,
// off-road, idle, the 8 nearest agents (into N.nb); returns the partial reward
__device__ __forceinline__ float lanes_events_a(const Slot& c, int lane, Agent& A, bool alive, float prevx,
                                                float prevy, float hx, float hy, const AgentQ* qp, int (&nb)[kK],
                                                uint32_t& ev, const Nbr& N) {
    float r = 0.f;
    if (alive) {
        const AgentQ q = *qp;
        A.step += 1;
        const float speed = sqrtf(A.vx * A.vx + A.vy * A.vy);
        if (q.seg >= 0) {
            float prog = (A.px - prevx) * q.tx + (A.py - prevy) * q.ty;
            r += kWProgress * clampf(prog, -kProgressClip, kProgressClip);
            float e = q.lat / kLaneSigma;
            float cosd = hx * q.tx + hy * q.ty;
            r += kWLane * (expf(-e * e) * ((1.f - kLaneWh) + kLaneWh * fmaxf(0.f, cosd)));
        }
        if (fabsf(q.lat) > kOffroadLat || q.dist > kOffroadDist) { ev |= kEvOffroad; r -= kWOffroad; }
        if (speed < kIdleSpeed) { ev |= kEvIdle; r -= kWIdle; }
#pragma unroll
        for (int t = 0; t < kK; ++t) nb[t] = N.nb[lane][t];   // the 8 nearest agents (pairs_knn)
    }
    return r;
}

// TTC and DRAC of every (slot, neighbour) pair of the block (all threads);
// the pair's own pose comes from the exchange area (published from the lane)
__device__ __forceinline__ void pairs_ttc_drac(const Exch& E, Nbr& N, int m, int tid, int nthreads) {
    for (int p = tid; p < m * kK; p += nthreads) {
        const int i = p / kK, t = p % kK, j = N.nb[i][t];
        if (j < 0) continue;
        N.tt[i][t] = ttc_pair(E.px[i], E.py[i], E.hx[i], E.hy[i], E.vx[i], E.vy[i], E.px[j], E.py[j], E.hx[j],
                              E.hy[j], E.vx[j], E.vy[j]);
        N.dr[i][t] = drac_pair(E.px[i], E.py[i], E.hx[i], E.hy[i], E.vx[i], E.vy[i], E.px[j], E.py[j], E.hx[j],
                               E.hy[j], E.vx[j], E.vy[j]);
    }
}

// events and rewards, second part: TTC / DRAC penalties, collision, edge,
// sparse events; done agents are marked for a respawn (auto-reset) or parked
// (coll_bits: the footprint overlaps found by pairs_knn, bit per slot)
__device__ __forceinline__ void lanes_events_b(const WorldArgs& args, int lane, Agent& A, bool& alive, bool nonfin,
                                               uint32_t coll_bits, const AgentQ* qp, const int (&nb)[kK],
                                               float (&tt)[kK], float r, const Nbr& N, uint32_t& ev, float& reward,
                                               float& drac, bool& done, bool& respawn, bool& parked_now) {
    if (alive) {
        const AgentQ q = *qp;
        float tmin = kTtcMax, dmax = 0.f;
#pragma unroll
        for (int t = 0; t < kK; ++t) {
            if (nb[t] < 0) continue;
            tt[t] = N.tt[lane][t];
            tmin = fminf(tmin, tt[t]);
            dmax = fmaxf(dmax, N.dr[lane][t]);
        }
        // App. G: p(tau) of the minimum TTC over the neighbours; a neighbour on no
        // collision course has TTC = tau_max (App. D), so any neighbour costs >= 0.01
        if (nb[0] >= 0) r -= penalty(kTtcAlphaV, tmin, kTtcPmaxV);
        r -= kWDrac * fmaxf(0.f, dmax - kDracThresh);
        drac = dmax;
        A.peak = fmaxf(A.peak, dmax);
        const bool collided = (coll_bits >> lane) & 1u;
        if (collided && A.step > kWarmup) ev |= kEvCollision;
        if (q.tedge < kInf) r -= penalty(kTtcAlphaE, q.tedge, kTtcPmaxE);
        if (q.forb) ev |= kEvLaneForb;
        float gdx = A.gx - A.px, gdy = A.gy - A.py;
        if (sqrtf(gdx * gdx + gdy * gdy) <= kGoalR) ev |= kEvGoal;
        float r22 = 1.f - 2.f * (A.qx * A.qx + A.qy * A.qy);
        float sdx = A.px - A.sx, sdy = A.py - A.sy;
        if (A.pz < 0.f || sqrtf(sdx * sdx + sdy * sdy) > kDriftMax || -r22 > kTiltGz) ev |= kEvCrash;
        if (ev & kEvGoal) r += kWGoal;
        else if (ev & kEvCollision) r -= kWCollision;
        else if (ev & kEvCrash) r -= kWCrash;
        else if (ev & kEvLaneForb) r -= kWLaneForb;
        if (A.step >= kMaxSteps) ev |= kEvTimeout;
        reward = r;
    }
    if (nonfin) { ev = kEvNonfinite; reward = 0.f; }
    const uint32_t sparse = kEvGoal | kEvCollision | kEvCrash | kEvLaneForb;
    const bool term = nonfin || (!(args.flags & kFlagInvincible) && (ev & sparse));
    done = term || (ev & kEvTimeout);
    if (done) {
        if (args.flags & kFlagAutoReset) respawn = true;
        else if (!nonfin) { park_agent(A); alive = false; parked_now = true; }
    }
}

// spawn candidates (x, y, psi, goal x, goal y, v0, candidate slot as int bits)
// of every try of every slot of a pack for the slot's next episode, drawn ahead
// of the respawns by threads t = 0..nt-1 (the draws depend on the slot, its
// episode and the try only)
constexpr int kSpawnDraws = 32 * kSpawnTries;
constexpr int kSpawnRows = 7;
constexpr int kSpawnGroup = 4;   // respawning slots whose tries are drawn together (one lane each)
__device__ __forceinline__ void draw_spawns(const WorldArgs& args, const int4& pk, const int* s_slot_w,
                                            const int* s_wbase, int t, int nt, float (*sp)[kSpawnDraws]) {
    for (int i = t; i < pk.w * kSpawnTries; i += nt) {
        const int j = i / kSpawnTries, r = i % kSpawnTries;
        const int wl = s_slot_w[j], a = pk.z + j;
        float x, y, psi, gx, gy, v0;
        int cs;
        spawn_candidate(args.rd, pk.x + wl, a, j - s_wbase[wl], args.st.episode[a] + 1, r, args.seed, x, y, psi, gx,
                        gy, v0, cs);
        sp[0][i] = x; sp[1][i] = y; sp[2][i] = psi; sp[3][i] = gx; sp[4][i] = gy; sp[5][i] = v0;
        sp[6][i] = __int_as_float(cs);
    }
}

// respawns of the marked lanes (App. J), every slot of the pack in index
// order, each spaced from the other alive agents of its own world.  A slot's
// kSpawnTries candidate draws depend on the slot, its episode and the try
// only, so they are read from `pre` (drawn ahead; may be null) or drawn for up
// to kSpawnGroup slots at once, one lane per (slot, try); the tries are then
// scored as a sequential loop would: the first one at least the spacing away
// is taken, else the one with the largest clearance (first on ties).
// spawn_slot (may be null) receives the respawned lane's spawn candidate slot.
// The clearances are taken over the positions in E.px / E.py, which this
// function sets to every lane's current position first (and each placed slot
// to its new one).
__device__ __forceinline__ void lanes_respawn(const WorldArgs& args, const Slot& c, int lane, Agent& A,
                                              bool& alive, bool respawn, uint32_t& ev, Exch& E,
                                              const float (*pre)[kSpawnDraws] = nullptr, int* spawn_slot = nullptr) {
    static_assert(kSpawnTries * kSpawnGroup == 32, "one lane per (slot, try) of a group");
    const uint32_t rbits = __ballot_sync(kFull, respawn);
    if (!rbits) return;
    E.px[lane] = A.px;
    E.py[lane] = A.py;
    __syncwarp();
    const unsigned long long seed = args.seed;
    const int q = lane / kSpawnTries, r = lane % kSpawnTries;
    for (uint32_t todo = rbits; todo;) {
        // the next kSpawnGroup respawning slots (ascending): lane (q, r) holds try r
        // of the group's q-th slot, read from `pre` or drawn here, all at once
        uint32_t group = 0u;
        for (int k = 0; k < kSpawnGroup && todo; ++k) {
            group |= todo & (~todo + 1u);
            todo &= todo - 1u;
        }
        uint32_t t = group;
        for (int k = 0; k < q && t; ++k) t &= t - 1u;
        const int lq = t ? __ffs(t) - 1 : 0;
        const int ep_q = __shfl_sync(kFull, A.episode, lq) + 1, w_q = __shfl_sync(kFull, c.w, lq);
        const int a_q = __shfl_sync(kFull, c.a, lq), base_q = __shfl_sync(kFull, c.base, lq);
        float x = 0.f, y = 0.f, psi = 0.f, gx = 0.f, gy = 0.f, v0 = 0.f;
        int cs = -1;
        if (t) {
            if (pre) {
                const int i = lq * kSpawnTries + r;
                x = pre[0][i]; y = pre[1][i]; psi = pre[2][i]; gx = pre[3][i]; gy = pre[4][i]; v0 = pre[5][i];
                cs = __float_as_int(pre[6][i]);
            } else {
                spawn_candidate(args.rd, w_q, a_q, lq - base_q, ep_q, r, seed, x, y, psi, gx, gy, v0, cs);
            }
        }
        // the group's slots in order: each takes the first try at least the spacing
        // away from every eligible agent, else the first of the largest clearance;
        // the eligible agents are the alive ones of its world, without the slots
        // still waiting to respawn.  Lane s0 + k holds try k of the g-th slot; the
        // tries are broadcast, lane j takes eligible agent j's squared distance to
        // each, and one warp minimum per try gives its clearance (a minimum of
        // squared distances >= +0: exact in any order, ordered like its bits).
        int g = 0;
        for (uint32_t gg = group; gg; gg &= gg - 1u, ++g) {
            const int l = __ffs(gg) - 1;
            const int ep = __shfl_sync(kFull, A.episode, l) + 1;
            const int lb = __shfl_sync(kFull, c.base, l), ln = __shfl_sync(kFull, c.n, l);
            const uint32_t wm = (ln >= 32 ? 0xFFFFFFFFu : ((1u << ln) - 1u)) << lb;
            const uint32_t later = l < 31 ? (rbits & (0xFFFFFFFFu << (l + 1))) : 0u;
            const uint32_t elig = __ballot_sync(kFull, alive) & wm & ~(1u << l) & ~later;
            const int s0 = g * kSpawnTries;
            const bool me = (elig >> lane) & 1u;
            const float ex = E.px[lane], ey = E.py[lane];
            unsigned dk[kSpawnTries];
#pragma unroll
            for (int k = 0; k < kSpawnTries; ++k) {
                const float tx = __shfl_sync(kFull, x, s0 + k), ty = __shfl_sync(kFull, y, s0 + k);
                dk[k] = __reduce_min_sync(kFull, me ? __float_as_uint(norm2(ex - tx, ey - ty)) : __float_as_uint(kInf));
            }
            const unsigned kClear = __float_as_uint(kSpawnSpacing * kSpawnSpacing);
            int pick = -1;
            unsigned best = 0u;
            int bk = 0;
#pragma unroll
            for (int k = 0; k < kSpawnTries; ++k) {
                if (pick < 0 && dk[k] >= kClear) pick = k;   // the first try clear of every agent
                if (dk[k] > best) { best = dk[k]; bk = k; }  // else the first of the largest clearance
            }
            const int src = s0 + (pick >= 0 ? pick : bk);
            const float bx = __shfl_sync(kFull, x, src), by = __shfl_sync(kFull, y, src);
            const float bpsi = __shfl_sync(kFull, psi, src), bv = __shfl_sync(kFull, v0, src);
            const float bgx = __shfl_sync(kFull, gx, src), bgy = __shfl_sync(kFull, gy, src);
            const int bcs = __shfl_sync(kFull, cs, src);
            if (lane == l) {
                place_agent(A, bx, by, bpsi, bv, bgx, bgy, (args.flags & kFlagWeatherAll) != 0);
                A.episode = ep;
                alive = true;
                ev |= kEvRespawned;
                if (spawn_slot) *spawn_slot = bcs;
                E.px[l] = A.px;
                E.py[l] = A.py;
            }
            __syncwarp();
        }
    }
}

// the final observation's neighbour tables get each slot's heading (lanes of
// the agent warp); the neighbours of the worlds that changed are recomputed
// by pairs_knn, and every lane then takes its row back into nb
__device__ __forceinline__ void lanes_final_a(int lane, float hx, float hy, Nbr& N) {
    N.hx[lane] = hx;
    N.hy[lane] = hy;
}

// neighbour rows of the observations (App. D analogue), one (slot, neighbour)
// pair per thread: 10 features relative to the slot's pose, zeros for an
// empty neighbour or a slot without an alive agent; TTC recomputed in a world
// that changed, else the events' value
__device__ __forceinline__ void pairs_nbr_rows(const WorldArgs& args, const Exch& E, const Nbr& N, int a0, int m,
                                               uint32_t alive_bits, uint32_t recompute_bits, uint32_t active_bits,
                                               int tid, int nthreads) {
    for (int p = tid; p < m * kK; p += nthreads) {
        const int i = p / kK, t = p % kK;
        if (!((active_bits >> i) & 1u)) continue;
        float s[10] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        const int j = N.nb[i][t];
        if (((alive_bits >> i) & 1u) && j >= 0) {
            const float hx = N.hx[i], hy = N.hy[i], px = E.px[i], py = E.py[i], vx = E.vx[i], vy = E.vy[i];
            const float pjx = E.px[j], pjy = E.py[j], hjx = E.hx[j], hjy = E.hy[j], vjx = E.vx[j], vjy = E.vy[j];
            float bx, by, dvx, dvy;
            to_ego(hx, hy, pjx - px, pjy - py, bx, by);
            to_ego(hx, hy, vjx - vx, vjy - vy, dvx, dvy);
            const float dpsi = atan2f(cross2(hx, hy, hjx, hjy), hx * hjx + hy * hjy);
            s[0] = bx / kSceneHalf;
            s[1] = by / kSceneHalf;
            s[2] = 2.f * kHalfLen / kSceneHalf;
            s[3] = 2.f * kHalfWid / kSceneHalf;
            s[4] = dpsi / 3.14159265358979323846f;
            s[5] = sqrtf(vjx * vjx + vjy * vjy) / 10.f;
            s[6] = dvx / 10.f;
            s[7] = dvy / 10.f;
            s[8] = (((recompute_bits >> i) & 1u) ? ttc_pair(px, py, hx, hy, vx, vy, pjx, pjy, hjx, hjy, vjx, vjy)
                                                  : N.tt[i][t]) / kTtcMax;
            s[9] = 1.f;
        }
        float2* row = reinterpret_cast<float2*>(args.out.obs + (size_t)(a0 + i) * kObsDim + kObsEgo + kObsNbr * t);
#pragma unroll
        for (int k = 0; k < 5; ++k) row[k] = make_float2(s[2 * k], s[2 * k + 1]);
    }
}

// ego group, outputs and state of the lanes of the agent warp
template <int MODE>
__device__ __forceinline__ void lanes_final_b(const WorldArgs& args, const Slot& c, int lane, Agent& A, bool alive,
                                              bool active, const AgentQ* qp, const int (&nb)[kK], float hx, float hy,
                                              uint32_t ev, float reward, bool done, float drac, bool respawn) {
    if (!(c.has && active)) return;
    const int a = c.a;
    float4* o4 = reinterpret_cast<float4*>(args.out.obs + (size_t)a * kObsDim);
    // an agent a reset did not move keeps its ego group and nearest lane
    const bool keep = MODE == kModeReset && alive && !respawn;
    AgentQ q;
    q.seg = -1;
    if (alive && !keep) {
        q = *qp;
        float gbx, gby, vbx, vby;
        to_ego(hx, hy, A.gx - A.px, A.gy - A.py, gbx, gby);
        to_ego(hx, hy, A.vx, A.vy, vbx, vby);
        float gn = sqrtf(gbx * gbx + gby * gby);
        uint32_t pc = A.meta & 0xFFu, sc = (A.meta >> 8) & 0xFFu;
        o4[0] = make_float4(gbx / kSceneHalf, gby / kSceneHalf, gn > 0.f ? gby / gn : 0.f, gn > 0.f ? gbx / gn : 1.f);
        o4[1] = make_float4(gn / kSceneHalf, vbx / 10.f, vby / 10.f,
                            weather_level(pc, (args.flags & kFlagWeatherAll) != 0));
        o4[2] = make_float4(sc == 0 ? 1.f : 0.f, sc == 1 ? 1.f : 0.f, sc == 2 ? 1.f : 0.f, A.wz);
        o4[3] = make_float4(A.dl / kThetaMax, A.mu, q.seg >= 0 ? q.lat / 3.6f : 0.f,
                            q.seg >= 0 ? cross2(q.tx, q.ty, hx, hy) : 0.f);
    } else if (!alive) {
#pragma unroll
        for (int k = 0; k < kObsEgo / 4; ++k) o4[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (args.flags & kFlagRecord) {
        if (!keep) args.out.lane_seg[a] = alive ? q.seg : -1;
#pragma unroll
        for (int t = 0; t < kK; ++t) args.out.knn_agents[(size_t)a * kK + t] = (alive && nb[t] >= 0) ? (a - lane) + nb[t] : -1;
    }
    if (MODE == kModeStep) {
        args.out.reward[a] = reward;
        args.out.done[a] = done ? 1 : 0;
        if (args.host_reward) {   // straight to the host buffers over the host link (posted stores)
            args.host_reward[a] = reward;
            args.host_done[a] = done ? 1 : 0;
        }
        args.out.events[a] = ev;
        args.out.drac[a] = drac;
    } else if (MODE == kModeReset && respawn) {
        args.out.events[a] = ev;
    }
    store_agent(args.st, a, A);
}

// ====================================================================== the fused world kernel
// One block per pack: consecutive worlds holding at most 32 agents together (one
// world per pack unless packing is enabled).  Warp 0 owns the agents (lane l =
// slot l = agent a0 + l): physics, events, respawns, neighbours, ego
// features, state; a lane only ever interacts with the slots of its own
// world.  All NW warps run the road queries, one agent per warp at a time, and
// write the road-point block of the observation with coalesced stores.
template <int MODE, int NW, int PHYS>
__global__ void __launch_bounds__(32 * NW, (16 / NW > 0 ? 16 / NW : 1)) world_kernel(const WorldArgs args) {
    __shared__ Exch E;
    __shared__ AgentQ Q[32];
    __shared__ Nbr N;
    __shared__ unsigned long long kbuf[NW][64];
    __shared__ unsigned s_alive, s_any, s_act, s_rec;
    __shared__ int s_slot_w[32];                  // pack-local world of each slot
    __shared__ int s_wbase[32], s_wn[32];         // per pack-local world: first slot, agents
    __shared__ int s_woff[32];                    // its blob's offset in s_blob, -1: read from global memory
    __shared__ DevGrid s_grid[32];
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ int s_staged;
    __shared__ float s_sp[kSpawnRows][kSpawnDraws];   // spawn candidates drawn ahead (kDraw)
    __shared__ int s_spawn[32];                   // spawn candidate slot of each respawned slot, -1: none
    __shared__ float s_d2[32][32];                // squared distances of the slot pairs (pairs_knn)
    __shared__ unsigned s_coll;                   // footprint overlap per slot (the collision event)
    __shared__ unsigned s_near[32];               // contact candidates of each slot (kDraw, step)
    extern __shared__ __align__(128) unsigned char s_blob[];
    // with spare warps, warps 1..NW-1 draw the spawn candidates of every slot
    // while warp 0 runs the physics (a step) or right after the masks (a reset),
    // so that the in-order respawns only pick among them
    constexpr bool kDraw = NW >= 4 && MODE != kModeObserve;
    // and, before the draws of a step, every slot's contact candidates (vehicle physics)
    constexpr bool kNear = kDraw && MODE == kModeStep && PHYS != kPhysBicycle;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int4 pk = __ldg(&args.packs[blockIdx.x]);   // (first world, worlds, first agent, agents)
    const int a0 = pk.z, m = pk.w;
    if (m <= 0) return;                               // CTA-uniform
    bool staged = false;                              // warp 0: this block copies its roads to shared memory
    int stage_total = 0;
    Agent A;
    float3 act = make_float3(0.f, 0.f, 0.f);
    if (warp == 0) {
        // lane l holds slot l = agent a0 + l: its state and actions are loaded
        // before the pack tables, so that the two memory round trips overlap
        const int al = a0 + (lane < m ? lane : 0);
        load_agent(args.st, al, A);
        if (MODE == kModeStep && lane < m) {
            const float* ap = args.actions + 3 * (size_t)al;
            act = make_float3(ap[0], ap[1], ap[2]);
        }
        pack_tables(args, pk, lane, s_slot_w, s_wbase, s_wn);
        int bytes = 0;
        if (lane < pk.y) {
            const DevGrid gg = args.rd.grid[pk.x + lane];
            s_grid[lane] = gg;
            bytes = gg.bytes;
        }
        int incl = bytes;                             // prefix sum of the blob sizes
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        stage_total = __shfl_sync(kFull, incl, 31);
        staged = args.stage_bytes > 0 && stage_total > 0 && stage_total <= args.stage_bytes;
        if (lane < pk.y) s_woff[lane] = staged ? incl - bytes : -1;
        if (lane == 0) s_staged = staged ? 1 : 0;
        __syncwarp();
        if (staged && MODE != kModeReset)
            stage_issue(args.rd.blob, s_grid, s_woff, pk.y, stage_total, s_blob, &s_bar, lane, args.withhold != 0);
        if (kDraw && MODE == kModeStep) named_bar_arrive(1, 32 * NW);   // the pack tables are written
    } else if (kDraw && MODE == kModeStep) {
        // the contact candidates for warp 0's physics, then the spawn draws
        float4 p = make_float4(0.f, 0.f, 0.f, 0.f), v = p;
        if (kNear) { p = args.st.pos[a0 + (lane < m ? lane : 0)]; v = args.st.vel[a0 + (lane < m ? lane : 0)]; }
        named_bar_sync(1, 32 * NW);
        if (kNear) {
            pairs_near(pk, s_slot_w, s_wbase, s_wn, warp - 1, NW - 1, lane, p.x, p.y,
                       cull_budget(v.x, v.y, args.h * args.substeps), s_near);
            named_bar_arrive(2, 32 * NW);
        }
        draw_spawns(args, pk, s_slot_w, s_wbase, threadIdx.x - 32, 32 * (NW - 1), s_sp);
    }

    // ---------------- warp 0: agent registers
    const Slot c = slot_of(pk, s_slot_w, s_wbase, s_wn, lane, warp == 0);
    bool alive = false, respawn = false, parked_now = false, nonfin = false, done = false;
    bool recompute = false, active = false;       // warp 0: neighbours recomputed / outputs written
    uint32_t ev = 0;
    float reward = 0.f, drac = 0.f, hx = 1.f, hy = 0.f;
    int nb[kK];
    float tt[kK];
#pragma unroll
    for (int t = 0; t < kK; ++t) { nb[t] = -1; tt[t] = kTtcMax; }
    if (warp == 0) {
        if (!c.has) A.meta = 0;
        alive = c.has && (status_of(A.meta) & kAlive);
        if (MODE == kModeReset) respawn = c.has && args.mask[c.a] != 0;
        const unsigned anyr = __ballot_sync(kFull, respawn);
        if (lane == 0) s_any = anyr;
    }
    if (MODE == kModeReset) {
        __syncthreads();
        if (s_any == 0u) return;                      // CTA-uniform: no masked agent in this pack
        if (warp == 0 && staged)
            stage_issue(args.rd.blob, s_grid, s_woff, pk.y, stage_total, s_blob, &s_bar, lane, args.withhold != 0);
        if (kDraw) {
            if (warp != 0) draw_spawns(args, pk, s_slot_w, s_wbase, threadIdx.x - 32, 32 * (NW - 1), s_sp);
            __syncthreads();
        }
    }
    bool stg = false;                                 // this thread reads the staged copies

    if (MODE == kModeStep) {
        float prevx = 0.f, prevy = 0.f;
        if (warp == 0) {
            lanes_physics<PHYS>(args, c, lane, A, alive, nonfin, prevx, prevy, hx, hy, E, act,
                                kNear ? s_near : nullptr, 32 * NW);
            const unsigned ab = __ballot_sync(kFull, alive);
            unsigned cb = 0u;
            if (NW == 1) {                            // a lane per slot: the per-lane forms
                __syncwarp();
                cb = __ballot_sync(kFull, lanes_knn(E, c.base, c.n, lane, ab, alive, true, N));
            }
            if (lane == 0) { s_alive = ab; s_coll = cb; }
        }
        __syncthreads();
        // ---------------- neighbours, footprint overlaps, TTC and DRAC at the end-of-physics
        // poses (all threads, pair-parallel)
        if (NW > 1) {
            const uint32_t slots = m >= 32 ? 0xFFFFFFFFu : ((1u << m) - 1u);
            pairs_knn(E, N, s_d2, s_slot_w, s_wbase, s_wn, m, s_alive, slots, &s_coll, threadIdx.x, 32 * NW);
            __syncthreads();
        }
        pairs_ttc_drac(E, N, m, threadIdx.x, 32 * NW);
        if (s_staged) {
            stg = stage_wait(&s_bar, args.wait_ns ? args.wait_ns : kStageWaitNs);
            if (!stg) atomicOr(args.out.error_word, 2u);
        }
        // ---------------- road queries at the end-of-physics pose (all warps, one agent at a
        // time), one pass over the cells: the events' answers and the observation's
        // road-point block (respawns and parking below replace the blocks they change)
        for (int j = warp; j < m; j += NW) {
            if (!((s_alive >> j) & 1u)) continue;
            const int t = s_slot_w[j];
            const WRoads v = view_of(s_grid[t], (stg && s_woff[t] >= 0) ? s_blob + s_woff[t]
                                                                         : args.rd.blob + s_grid[t].blob);
            float* hnt = args.out.hint + 4 * (size_t)(a0 + j);
            const float4 h4 = *reinterpret_cast<const float4*>(hnt);
            const float hv[4] = {h4.x, h4.y, h4.z, h4.w};
            const AgentQ q = agent_step_queries<true>(
                v, E.px[j], E.py[j], E.gx[j], E.gy[j], E.hx[j], E.hy[j], E.vx[j], E.vy[j], hv, hnt, lane, kbuf[warp],
                args.out.obs + (size_t)(a0 + j) * kObsDim + kObsEgo + kK * kObsNbr,
                (args.flags & kFlagRecord) ? args.out.knn_pts + (size_t)(a0 + j) * kL : nullptr);
            if (lane == 0) Q[j] = q;
        }
        __syncthreads();
        // ---------------- events and rewards (App. G), lanes of the agent warp
        if (warp == 0) {
            const float r = lanes_events_a(c, lane, A, alive, prevx, prevy, hx, hy, &Q[lane], nb, ev, N);
            lanes_events_b(args, lane, A, alive, nonfin, s_coll, &Q[lane], nb, tt, r, N, ev, reward, drac, done,
                           respawn, parked_now);
        }
    }

    // ---------------- respawns (warp 0, agents in index order), then the post-reset exchange
    if (warp == 0) {
        int spawn_slot = -1;
        lanes_respawn(args, c, lane, A, alive, respawn, ev, E, kDraw ? s_sp : nullptr, &spawn_slot);
        s_spawn[lane] = respawn ? spawn_slot : -1;
        // per world (never per pack, so that packing changes no result): a world
        // with a respawn or a parked agent republishes and recomputes its
        // neighbours; a reset leaves the worlds without a masked agent untouched
        const unsigned chg = __ballot_sync(kFull, respawn || parked_now);
        const uint32_t wmask = c.n >= 32 ? 0xFFFFFFFFu : (((1u << c.n) - 1u) << c.base);
        const bool wchanged = (chg & wmask) != 0u;
        recompute = (MODE != kModeStep) || wchanged;
        active = (MODE != kModeReset) || wchanged;
        heading_of(A.qw, A.qx, A.qy, A.qz, hx, hy);
        __syncwarp();
        if (recompute) publish(E, lane, A, hx, hy);
        const unsigned ab = __ballot_sync(kFull, alive), act = __ballot_sync(kFull, active);
        if (lane == 0) { s_alive = ab; s_act = act; }
        // road-point blocks to compute: every agent when observing, the respawned
        // ones otherwise (the step's queries wrote the others' at the same pose;
        // a reset moves only its masked agents, so the others' blocks and ego
        // groups stand)
        if (lane < m) Q[lane].need = (MODE == kModeObserve || respawn) ? 1 : 0;
    }
    __syncthreads();

    // ---------------- road-point block of every observation (all warps)
    if (MODE != kModeStep && s_staged) {
        stg = stage_wait(&s_bar, args.wait_ns ? args.wait_ns : kStageWaitNs);
        if (!stg) atomicOr(args.out.error_word, 2u);
    }
    for (int j = warp; j < m; j += NW) {
        if (!((s_act >> j) & 1u)) continue;
        const int t = s_slot_w[j];
        const WRoads v = view_of(s_grid[t], (stg && s_woff[t] >= 0) ? s_blob + s_woff[t]
                                                                     : args.rd.blob + s_grid[t].blob);
        const bool al = (s_alive >> j) & 1u, need = Q[j].need != 0;
        if (MODE != kModeObserve && al && !need) continue;   // written by the step's queries / unmoved by the reset
        float* orow = args.out.obs + (size_t)(a0 + j) * kObsDim + kObsEgo + kK * kObsNbr;
        int32_t* krow = (args.flags & kFlagRecord) ? args.out.knn_pts + (size_t)(a0 + j) * kL : nullptr;
        float* hnt = args.out.hint + 4 * (size_t)(a0 + j);
        const int slot = MODE != kModeObserve ? s_spawn[j] : -1;
        Lane L;
        if (al && need && slot >= 0 && args.rd.spawnq)      // a respawn on a spawn candidate: the table's answers
            spawn_road_block(args.rd.spawnq + slot, v, E.px[j], E.py[j], E.gx[j], E.gy[j], E.hx[j], E.hy[j], hnt,
                             lane, orow, krow, &L);
        else
            agent_road_block<true>(v, al, need, E.px[j], E.py[j], E.gx[j], E.gy[j], E.hx[j], E.hy[j], hnt, lane,
                             kbuf[warp], orow, krow, &L, MODE == kModeObserve ? kLaneR0 : kSpawnLaneR);
        if (al && need && lane == 0) {
            Q[j].seg = L.seg; Q[j].dist = L.dist; Q[j].lat = L.lat; Q[j].tx = L.tx; Q[j].ty = L.ty;
        }
    }
    __syncthreads();

    // ---------------- neighbours of the worlds that changed (all threads), their rows (all
    // warps), ego group, outputs, state (warp 0)
    if (warp == 0) {
        // no copy may outlive the block: after a wait that gave up, wait again
        // (bounded by 1 s whatever the caller's limit) for the copy this block issued
        if (lane == 0 && s_staged && !stg && !args.withhold) stage_wait(&s_bar, kStageWaitNs);
        lanes_final_a(lane, hx, hy, N);
        if (NW == 1 && recompute) lanes_knn(E, c.base, c.n, lane, s_alive, alive, false, N);
        const unsigned rb = __ballot_sync(kFull, recompute);
        if (lane == 0) s_rec = rb;
    }
    __syncthreads();
    if (NW > 1 && s_rec) {                            // CTA-uniform
        pairs_knn(E, N, s_d2, s_slot_w, s_wbase, s_wn, m, s_alive, s_rec, nullptr, threadIdx.x, 32 * NW);
        __syncthreads();
    }
    pairs_nbr_rows(args, E, N, a0, m, s_alive, s_rec, s_act, threadIdx.x, 32 * NW);
    if (warp != 0) return;
    if (recompute) {
#pragma unroll
        for (int t = 0; t < kK; ++t) nb[t] = N.nb[lane][t];
    }
    lanes_final_b<MODE>(args, c, lane, A, alive, active, &Q[lane], nb, hx, hy, ev, reward, done, drac, respawn);
}

// ====================================================================== the split step
// The same step as four kernels: the lane-per-agent phases (physics; events,
// respawns and the ego / neighbour groups) run one warp per pack, the road
// queries one warp per agent in blocks of NWQ warps, so that the query kernels
// keep a small register footprint and many warps resident.  Results are
// bit-identical to the fused kernel (the same inline code).

// physics; writes the state, the start-of-step position, the heading and the
// non-finite flag
template <int PHYS>
__global__ void __launch_bounds__(32, 16) phys_kernel(const WorldArgs args) {
    __shared__ Exch E;
    __shared__ int s_slot_w[32], s_wbase[32], s_wn[32];
    const int lane = threadIdx.x;
    const int4 pk = __ldg(&args.packs[blockIdx.x]);
    if (pk.w <= 0) return;
    pack_tables(args, pk, lane, s_slot_w, s_wbase, s_wn);
    const Slot c = slot_of(pk, s_slot_w, s_wbase, s_wn, lane, true);
    Agent A;
    load_agent(args.st, c.a, A);
    float3 act = make_float3(0.f, 0.f, 0.f);
    if (c.has) {
        const float* ap = args.actions + 3 * (size_t)c.a;
        act = make_float3(ap[0], ap[1], ap[2]);
    }
    if (!c.has) A.meta = 0;
    bool alive = c.has && (status_of(A.meta) & kAlive), nonfin = false;
    float prevx = 0.f, prevy = 0.f, hx = 1.f, hy = 0.f;
    if (blockIdx.x == 0 && lane == 0) *args.sc.fix_count = 0u;   // the events kernel appends after this kernel
    lanes_physics<PHYS>(args, c, lane, A, alive, nonfin, prevx, prevy, hx, hy, E, act);
    if (c.has) {
        store_agent(args.st, c.a, A);
        args.sc.prev[c.a] = make_float2(prevx, prevy);
        args.sc.head[c.a] = make_float2(hx, hy);
        args.sc.flag[c.a] = nonfin ? 1 : 0;
    }
}

// road queries of one agent per warp: the events' queries (into sc.q) and the
// road-point block of the observation at the post-physics pose
template <int NWQ>
__global__ void __launch_bounds__(32 * NWQ, 32 / NWQ) query_kernel(const WorldArgs args) {
    __shared__ unsigned long long kbuf[NWQ][64];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int a = blockIdx.x * NWQ + warp;
    if (a >= args.num_agents) return;                 // warp-uniform
    float* orow = args.out.obs + (size_t)a * kObsDim + kObsEgo + kK * kObsNbr;
    int32_t* krow = (args.flags & kFlagRecord) ? args.out.knn_pts + (size_t)a * kL : nullptr;
    // every per-agent load at once (one memory round trip), then the world's grid
    const uint32_t meta = args.st.meta[a];
    const int wid = args.sc.agent_world[a];
    const float4 p = args.st.pos[a], vel = args.st.vel[a], goal = args.st.goal[a];
    const float2 h = args.sc.head[a];
    float* hnt = args.out.hint + 4 * (size_t)a;
    const float4 h4 = *reinterpret_cast<const float4*>(hnt);
    if (!(status_of(meta) & kAlive)) {
#pragma unroll
        for (int k = 0; k < kObsPt; ++k) orow[kObsPt * lane + k] = 0.f;
        if (krow) krow[lane] = -1;
        return;
    }
    const DevGrid g = args.rd.grid[wid];
    const WRoads v = view_of(g, args.rd.blob + g.blob);
    const float hv[4] = {h4.x, h4.y, h4.z, h4.w};
    const AgentQ q = agent_step_queries<false>(v, p.x, p.y, goal.x, goal.y, h.x, h.y, vel.x, vel.y, hv, hnt, lane,
                                        kbuf[warp], orow, krow);
    if (lane == 0) args.sc.q[a] = q;
}

// events, rewards, respawns, neighbours, ego group, outputs and state; marks
// the agents whose road-point block is stale (respawned or parked).  Warp 0
// holds the agents; the (agent, neighbour) pairs are spread over NWE warps.
template <int NWE>
__global__ void __launch_bounds__(32 * NWE) events_kernel(const WorldArgs args) {
    __shared__ Exch E;
    __shared__ Nbr N;
    __shared__ int s_slot_w[32], s_wbase[32], s_wn[32];
    __shared__ unsigned s_alive, s_rec, s_coll;
    __shared__ float s_d2[32][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int4 pk = __ldg(&args.packs[blockIdx.x]);
    const int m = pk.w;
    if (m <= 0) return;
    if (warp == 0) pack_tables(args, pk, lane, s_slot_w, s_wbase, s_wn);
    __syncthreads();
    const Slot c = slot_of(pk, s_slot_w, s_wbase, s_wn, lane, warp == 0);
    Agent A;
    bool alive = false, nonfin = false, respawn = false, parked_now = false, done = false, recompute = false;
    float prevx = 0.f, prevy = 0.f, hx = 1.f, hy = 0.f, reward = 0.f, drac = 0.f, r = 0.f;
    uint32_t ev = 0, alive_bits = 0;
    int nb[kK];
    float tt[kK];
#pragma unroll
    for (int t = 0; t < kK; ++t) { nb[t] = -1; tt[t] = kTtcMax; }
    if (warp == 0) {
        load_agent(args.st, c.a, A);
        if (!c.has) A.meta = 0;
        alive = c.has && (status_of(A.meta) & kAlive);
        nonfin = c.has && (args.sc.flag[c.a] & 1u);
        if (c.has) {
            const float2 pv = args.sc.prev[c.a], hd = args.sc.head[c.a];
            prevx = pv.x; prevy = pv.y; hx = hd.x; hy = hd.y;
        }
        publish(E, lane, A, hx, hy);
        alive_bits = __ballot_sync(kFull, alive);
        unsigned cb = 0u;
        if (NWE == 1) {                               // a lane per slot: the per-lane forms
            __syncwarp();
            cb = __ballot_sync(kFull, lanes_knn(E, c.base, c.n, lane, alive_bits, alive, true, N));
        }
        if (lane == 0) { s_alive = alive_bits; s_coll = cb; }
    }
    __syncthreads();
    if (NWE > 1) {                                    // pair-parallel over the block's warps
        const uint32_t slots = m >= 32 ? 0xFFFFFFFFu : ((1u << m) - 1u);
        pairs_knn(E, N, s_d2, s_slot_w, s_wbase, s_wn, m, s_alive, slots, &s_coll, threadIdx.x, 32 * NWE);
        __syncthreads();
    }
    pairs_ttc_drac(E, N, m, threadIdx.x, 32 * NWE);
    __syncthreads();
    if (warp == 0) {
        r = lanes_events_a(c, lane, A, alive, prevx, prevy, hx, hy, args.sc.q + c.a, nb, ev, N);
        lanes_events_b(args, lane, A, alive, nonfin, s_coll, args.sc.q + c.a, nb, tt, r, N, ev, reward, drac, done,
                       respawn, parked_now);
        lanes_respawn(args, c, lane, A, alive, respawn, ev, E);
        const unsigned chg = __ballot_sync(kFull, respawn || parked_now);
        const uint32_t wmask = c.n >= 32 ? 0xFFFFFFFFu : (((1u << c.n) - 1u) << c.base);
        recompute = (chg & wmask) != 0u;
        heading_of(A.qw, A.qx, A.qy, A.qz, hx, hy);
        __syncwarp();
        if (recompute) publish(E, lane, A, hx, hy);
        const uint32_t alive_now = __ballot_sync(kFull, alive);
        __syncwarp();
        if (c.has) {
            args.sc.head[c.a] = make_float2(hx, hy);
            args.sc.flag[c.a] = (respawn || parked_now) ? 2 : 0;
            if (respawn || parked_now) args.sc.fix_list[atomicAdd(args.sc.fix_count, 1u)] = c.a;
        }
        lanes_final_a(lane, hx, hy, N);
        if (NWE == 1 && recompute) lanes_knn(E, c.base, c.n, lane, alive_now, alive, false, N);
        const unsigned rb = __ballot_sync(kFull, recompute);
        if (lane == 0) { s_alive = alive_now; s_rec = rb; }
    }
    __syncthreads();
    if (NWE > 1 && s_rec) {                           // CTA-uniform
        pairs_knn(E, N, s_d2, s_slot_w, s_wbase, s_wn, m, s_alive, s_rec, nullptr, threadIdx.x, 32 * NWE);
        __syncthreads();
    }
    pairs_nbr_rows(args, E, N, pk.z, m, s_alive, s_rec, 0xFFFFFFFFu, threadIdx.x, 32 * NWE);
    if (warp != 0) return;
    if (recompute) {
#pragma unroll
        for (int t = 0; t < kK; ++t) nb[t] = N.nb[lane][t];
    }
    lanes_final_b<kModeStep>(args, c, lane, A, alive, true, args.sc.q + c.a, nb, hx, hy, ev, reward, done, drac,
                             respawn);
}

// road-point blocks of the agents the events kernel respawned (nearest lane
// and 32 points from the default radii, the ego lane features) or parked
// (zeros): the warps of a small grid walk the events kernel's list
template <int NWQ>
__global__ void __launch_bounds__(32 * NWQ) fix_kernel(const WorldArgs args) {
    __shared__ unsigned long long kbuf[NWQ][64];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned count = *args.sc.fix_count;
    for (unsigned i = blockIdx.x * NWQ + warp; i < count; i += gridDim.x * NWQ) {   // warp-uniform
        const int a = args.sc.fix_list[i];
        float* orow = args.out.obs + (size_t)a * kObsDim + kObsEgo + kK * kObsNbr;
        int32_t* krow = (args.flags & kFlagRecord) ? args.out.knn_pts + (size_t)a * kL : nullptr;
        if (!(status_of(args.st.meta[a]) & kAlive)) {
#pragma unroll
            for (int k = 0; k < kObsPt; ++k) orow[kObsPt * lane + k] = 0.f;
            if (krow) krow[lane] = -1;
            continue;
        }
        const DevGrid g = args.rd.grid[args.sc.agent_world[a]];
        const WRoads v = view_of(g, args.rd.blob + g.blob);
        const float4 p = args.st.pos[a], goal = args.st.goal[a];
        const float2 h = args.sc.head[a];
        Lane L;
        agent_road_block<false>(v, true, true, p.x, p.y, goal.x, goal.y, h.x, h.y, args.out.hint + 4 * (size_t)a, lane,
                         kbuf[warp], orow, krow, &L, kSpawnLaneR);
        if (lane == 0) {
            float* ego = args.out.obs + (size_t)a * kObsDim;
            ego[14] = L.seg >= 0 ? L.lat / 3.6f : 0.f;
            ego[15] = L.seg >= 0 ? cross2(L.tx, L.ty, h.x, h.y) : 0.f;
            if (args.flags & kFlagRecord) args.out.lane_seg[a] = L.seg;
        }
        __syncwarp();
    }
}

// explicit placement: d_place[a] = (x, y, psi, v0, gx, gy)
__global__ void place_kernel(const WorldArgs args, const float* __restrict__ place) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= args.num_agents) return;
    Agent A;
    load_agent(args.st, a, A);
    const float* p = place + 6 * (size_t)a;
    place_agent(A, p[0], p[1], p[2], p[3], p[4], p[5], (args.flags & kFlagWeatherAll) != 0);
    store_agent(args.st, a, A);
}

// gate per agent, one warp per world
__global__ void surr_gate_kernel(const WorldArgs args, float dt, uint8_t* __restrict__ elig) {
    __shared__ Exch E;
    const int w = blockIdx.x, lane = threadIdx.x;
    const int4 wd = __ldg(&args.rd.world[w]);
    const int a0 = wd.x, n = wd.y;
    if (n <= 0) return;
    const bool has = lane < n;
    const int a = a0 + (has ? lane : 0);
    Agent A;
    load_agent(args.st, a, A);
    const bool alive = has && (status_of(A.meta) & kAlive);
    float hx, hy;
    heading_of(A.qw, A.qx, A.qy, A.qz, hx, hy);
    publish(E, lane, A, hx, hy);
    const uint32_t ab = __ballot_sync(kFull, alive);
    __syncwarp();
    const bool g = surr_gate(E, 0, n, lane, ab, A, dt);
    if (has) elig[a] = g ? 1 : 0;
}

__global__ void surr_features_kernel(const WorldArgs args, const float* __restrict__ actions,
                                     const float* __restrict__ stats, float* __restrict__ x) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= args.num_agents) return;
    Agent A;
    load_agent(args.st, a, A);
    const float* act = actions + 3 * (size_t)a;
    float f[kSurrIn];
    surr_features(A, clampf(act[0], 0.f, 1.f), kThetaMax * clampf(act[1], -1.f, 1.f), clampf(act[2], 0.f, 1.f), f);
    float* row = x + (size_t)a * kSurrInLd;
#pragma unroll
    for (int k = 0; k < kSurrIn; ++k) row[k] = stats ? (f[k] - stats[k]) / stats[kSurrIn + k] : f[k];
    row[30] = 0.f;
    row[31] = 0.f;
}

__global__ void surr_snapshot_kernel(const WorldArgs args, float4* __restrict__ snap) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    const int A = args.num_agents;
    if (a >= A) return;
    snap[a] = args.st.pos[a];
    snap[A + a] = args.st.quat[a];
    snap[2 * A + a] = args.st.vel[a];
    snap[3 * A + a] = args.st.angv[a];
    snap[4 * A + a] = args.st.spin[a];
}

// One block walks the agents in order, kCollectThreads at a time, and gives
// each kept transition the next row: row i of the training set is the i-th
// kept transition in (step, agent) order, so the rows, the normalisation
// fitted to them and the trained weights repeat from run to run (an atomic
// ticket per row would order them by scheduling).
constexpr int kCollectThreads = 512;

__global__ void __launch_bounds__(kCollectThreads, 1)
    surr_collect_kernel(const WorldArgs args, const float4* __restrict__ snap, const uint8_t* __restrict__ elig,
                        const float* __restrict__ x, float dt, float* __restrict__ out_x, float* __restrict__ out_y,
                        unsigned long long cap, unsigned long long* __restrict__ count) {
    __shared__ unsigned s_cnt[kCollectThreads / 32];
    __shared__ unsigned long long s_base;
    const int A = args.num_agents;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_base = *count;
    __syncthreads();
    unsigned long long base = s_base;
    for (int a0 = 0; a0 < A; a0 += kCollectThreads) {
        const int a = a0 + (int)threadIdx.x;
        bool keep = false;
        float y[kSurrOut];
        if (a < A && elig[a] &&
            !(args.out.events[a] & (kEvRespawned | kEvNonfinite | kEvCollision | kEvCrash))) {
            Agent S;
            load_agent(args.st, a, S);
            if (status_of(S.meta) & kAlive) {
                keep = true;
                surr_targets(snap[a], snap[A + a], snap[2 * A + a], snap[3 * A + a], snap[4 * A + a], S, dt, y);
            }
        }
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) s_cnt[w] = __popc(m);
        __syncthreads();
        unsigned before = 0, total = 0;
#pragma unroll
        for (int j = 0; j < kCollectThreads / 32; ++j) {
            const unsigned c = s_cnt[j];
            before += j < w ? c : 0u;
            total += c;
        }
        __syncthreads();
        if (keep) {
            const unsigned long long i = base + before + __popc(m & ((1u << lane) - 1u));
            if (i < cap) {
#pragma unroll
                for (int k = 0; k < kSurrIn; ++k) out_x[i * kSurrIn + k] = x[(size_t)a * kSurrInLd + k];
#pragma unroll
                for (int k = 0; k < kSurrOut; ++k) out_y[i * kSurrOut + k] = y[k];
            }
        }
        base += total;
    }
    if (threadIdx.x == 0) *count = base;
}

cudaError_t sf_launch_surr_gate(const WorldArgs& a, float dt, uint8_t* d_elig, cudaStream_t s) {
    if (a.num_worlds <= 0) return cudaSuccess;
    surr_gate_kernel<<<a.num_worlds, 32, 0, s>>>(a, dt, d_elig);
    return cudaGetLastError();
}
cudaError_t sf_launch_surr_features(const WorldArgs& a, const float* d_actions, const float* x_stats, float* d_x,
                                    cudaStream_t s) {
    if (a.num_agents <= 0) return cudaSuccess;
    surr_features_kernel<<<(a.num_agents + 127) / 128, 128, 0, s>>>(a, d_actions, x_stats, d_x);
    return cudaGetLastError();
}
cudaError_t sf_launch_surr_snapshot(const WorldArgs& a, float4* snap, cudaStream_t s) {
    if (a.num_agents <= 0) return cudaSuccess;
    surr_snapshot_kernel<<<(a.num_agents + 127) / 128, 128, 0, s>>>(a, snap);
    return cudaGetLastError();
}
cudaError_t sf_launch_surr_collect(const WorldArgs& a, const float4* snap, const uint8_t* d_elig, const float* d_x,
                                   float dt, float* out_x, float* out_y, unsigned long long cap,
                                   unsigned long long* count, cudaStream_t s) {
    if (a.num_agents <= 0) return cudaSuccess;
    surr_collect_kernel<<<1, kCollectThreads, 0, s>>>(a, snap, d_elig, d_x, dt, out_x, out_y, cap, count);
    return cudaGetLastError();
}

template <int NWQ>
static cudaError_t launch_split(const WorldArgs& a, cudaStream_t s) {
    const int qb = (a.num_agents + NWQ - 1) / NWQ;
    switch (phys_of(a)) {
        case kPhysBicycle: phys_kernel<kPhysBicycle><<<a.num_packs, 32, 0, s>>>(a); break;
        case kPhysSurrogate: phys_kernel<kPhysSurrogate><<<a.num_packs, 32, 0, s>>>(a); break;
        default: phys_kernel<kPhysVehicle><<<a.num_packs, 32, 0, s>>>(a); break;
    }
    query_kernel<NWQ><<<qb, 32 * NWQ, 0, s>>>(a);
    // blocks of about 32 agents keep one warp for their pairs (more blocks
    // resident); blocks of one small world spread them over four
    if (a.num_agents > 16 * a.num_packs) events_kernel<1><<<a.num_packs, 32, 0, s>>>(a);
    else events_kernel<4><<<a.num_packs, 128, 0, s>>>(a);
    fix_kernel<NWQ><<<min(qb, 4 * 148), 32 * NWQ, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t sf_launch_step_split(const WorldArgs& a, int nwq, cudaStream_t s) {
    if (a.num_packs <= 0 || a.num_agents <= 0) return cudaSuccess;
    switch (nwq) {
        case 2: return launch_split<2>(a, s);
        case 8: return launch_split<8>(a, s);
        default: return launch_split<4>(a, s);
    }
}

template <int MODE, int NW, int PHYS>
static cudaError_t launch_shape(const WorldArgs& a, cudaStream_t s) {
    // allow up to kMaxStageBytes of dynamic shared memory, once per instantiation
    static const cudaError_t attr = cudaFuncSetAttribute(world_kernel<MODE, NW, PHYS>,
                                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxStageBytes);
    if (attr != cudaSuccess) return attr;
    if (a.stage_bytes < 0 || a.stage_bytes > kMaxStageBytes || a.stage_bytes % 16) return cudaErrorInvalidValue;
    world_kernel<MODE, NW, PHYS><<<a.num_packs, 32 * NW, a.stage_bytes, s>>>(a);
    return cudaGetLastError();
}

template <int MODE, int PHYS>
static cudaError_t launch_nw(const WorldArgs& a, int nw, cudaStream_t s) {
    switch (nw) {
        case 1: return launch_shape<MODE, 1, PHYS>(a, s);
        case 2: return launch_shape<MODE, 2, PHYS>(a, s);
        case 8: return launch_shape<MODE, 8, PHYS>(a, s);
        default: return launch_shape<MODE, 4, PHYS>(a, s);
    }
}

// a step's kernel carries only its physics variant; resets and observations run none
template <int MODE>
static cudaError_t launch_mode(const WorldArgs& a, int nw, cudaStream_t s) {
    if (MODE != kModeStep) return launch_nw<MODE, kPhysVehicle>(a, nw, s);
    switch (phys_of(a)) {
        case kPhysBicycle: return launch_nw<MODE, kPhysBicycle>(a, nw, s);
        case kPhysSurrogate: return launch_nw<MODE, kPhysSurrogate>(a, nw, s);
        default: return launch_nw<MODE, kPhysVehicle>(a, nw, s);
    }
}

cudaError_t sf_launch_world(int mode, const WorldArgs& a, int nw, cudaStream_t s) {
    if (a.num_packs <= 0) return cudaSuccess;
    switch (mode) {
        case kModeStep: return launch_mode<kModeStep>(a, nw, s);
        case kModeReset: return launch_mode<kModeReset>(a, nw, s);
        default: return launch_mode<kModeObserve>(a, nw, s);
    }
}

// the spawn table: per spawn candidate (one warp each) the exact nearest lane
// (before the goal orientation) and the 32 nearest road points at the
// candidate point, by the same queries the step runs
__global__ void __launch_bounds__(256) spawn_table_kernel(const DevRoads rd, const int32_t* __restrict__ cand_world,
                                                          int ncand, SpawnQ* __restrict__ out) {
    __shared__ unsigned long long kbuf[8][64];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x * 8 + warp;
    if (c >= ncand) return;                           // warp-uniform
    const DevGrid g = rd.grid[cand_world[c]];
    const WRoads v = view_of(g, rd.blob + g.blob);
    const float4 p = rd.pt[rd.cands[c]];
    const unsigned long long key = coop_knn32<false>(v, p.x, p.y, kKnnR0, lane, kbuf[warp]);
    __syncwarp();
    const Lane L = coop_nearest_lane_raw(v, p.x, p.y, kSpawnLaneR, lane);
    const unsigned long long last = shfl64(key, 31);
    SpawnQ* e = out + c;
    e->pos[lane] = key != kKeyInf ? (uint16_t)rkey_pos(key) : (uint16_t)0xFFFFu;
    if (lane == 0) {
        e->seg = L.seg; e->dist = L.dist; e->lat = L.lat; e->tx = L.tx; e->ty = L.ty;
        e->d32 = last != kKeyInf ? sqrtf(key_d2(last)) : 0.f;
        e->pad[0] = e->pad[1] = 0;
    }
}

cudaError_t sf_launch_spawn_table(const DevRoads& rd, const int32_t* cand_world, int ncand, SpawnQ* out,
                                  cudaStream_t s) {
    if (ncand <= 0) return cudaSuccess;
    spawn_table_kernel<<<(ncand + 7) / 8, 256, 0, s>>>(rd, cand_world, ncand, out);
    return cudaGetLastError();
}

cudaError_t sf_launch_place(const WorldArgs& a, const float* d_place, cudaStream_t s) {
    if (a.num_agents <= 0) return cudaSuccess;
    place_kernel<<<(a.num_agents + 127) / 128, 128, 0, s>>>(a, d_place);
    return cudaGetLastError();
}

// ====================================================================== the full observation (App. D)
// One warp per agent.  Ego group and weather token; road context: the world's
// segment midpoints within 10 m, scanned in ascending point index (polyline
// order) 32 at a time, each lane testing one midpoint, a ballot and a prefix
// count placing the hits in order, stopping once 350 slots are filled;
// neighbour context: a bitonic sort of the (squared distance, index) keys of
// the world's other alive agents, one lane per slot.  Every slot that is not
// filled is written as zeros, so the row is complete after the call.
template <int NW>
__global__ void __launch_bounds__(32 * NW) full_obs_kernel(const FullObsArgs f) {
    const int lane = threadIdx.x & 31;
    const int a = blockIdx.x * NW + (threadIdx.x >> 5);
    if (a >= f.num_agents) return;
    float* o = f.obs + (size_t)a * kFullObs;
    const uint32_t meta = f.st.meta[a];
    if (!(status_of(meta) & kAlive)) {
        for (int i = lane; i < kFullObs; i += 32) o[i] = 0.f;
        if (lane == 0) {
            if (f.n_road) f.n_road[a] = 0;
            if (f.n_veh) f.n_veh[a] = 0;
        }
        if (f.road_idx) for (int t = lane; t < kFullKR; t += 32) f.road_idx[(size_t)a * kFullKR + t] = -1;
        if (f.veh_idx && lane < kFullKV) f.veh_idx[(size_t)a * kFullKV + lane] = -1;
        return;
    }
    const float4 p = f.st.pos[a], q = f.st.quat[a], v = f.st.vel[a], g = f.st.goal[a];
    float hx, hy;
    heading_of(q.x, q.y, q.z, q.w, hx, hy);

    // ---- ego group (11)
    {
        float gbx, gby, vbx, vby;
        to_ego(hx, hy, g.x - p.x, g.y - p.y, gbx, gby);
        to_ego(hx, hy, v.x, v.y, vbx, vby);
        const float gn = sqrtf(gbx * gbx + gby * gby);
        const uint32_t pc = meta & 0xFFu, sc = (meta >> 8) & 0xFFu;
        float e = 0.f;
        switch (lane) {
            case 0: e = gbx / kSceneHalf; break;
            case 1: e = gby / kSceneHalf; break;
            case 2: e = gn > 0.f ? gby / gn : 0.f; break;
            case 3: e = gn > 0.f ? gbx / gn : 1.f; break;
            case 4: e = gn / kSceneHalf; break;
            case 5: e = vbx / 10.f; break;
            case 6: e = vby / 10.f; break;
            case 7: e = weather_level(pc, f.weather_all != 0); break;
            case 8: e = sc == 0 ? 1.f : 0.f; break;
            case 9: e = sc == 1 ? 1.f : 0.f; break;
            case 10: e = sc == 2 ? 1.f : 0.f; break;
            default: break;
        }
        if (lane < kFullEgo) o[lane] = e;
    }

    // ---- road context (350 x 5)
    const int w = f.agent_world[a];
    const int4 wd = f.rd.world[w];   // first agent, agents, first point, points
    const int kend = wd.z + wd.w;
    int nr = 0;
    // four chunks of 32 midpoints (and their types) are loaded before any is used: memory-level
    // parallelism for a scan whose every step otherwise waits on one L2 round trip
    for (int base = wd.z; base < kend && nr < kFullKR; base += 128) {
        float4 m[4];
        uint32_t ty[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int k = base + 32 * u + lane;
            m[u] = k < kend ? __ldg(f.rd.mid + k) : make_float4(kInf, 0.f, 0.f, 0.f);
            ty[u] = k < kend ? (uint32_t)__ldg(f.rd.ptype + k) : 0u;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int k = base + 32 * u + lane;
            const float dx = m[u].x - p.x, dy = m[u].y - p.y;
            const bool in = dx * dx + dy * dy <= kFullR2;
            const unsigned bal = __ballot_sync(kFull, in);
            const int slot = nr + __popc(bal & ((1u << lane) - 1u));
            if (in && slot < kFullKR) {
                float bx, by, ux, uy;
                to_ego(hx, hy, dx, dy, bx, by);
                to_ego(hx, hy, m[u].z, m[u].w, ux, uy);
                float* s = o + kFullRoad0 + kFullPt * slot;
                s[0] = bx / 10.f;
                s[1] = by / 10.f;
                s[2] = (float)ty[u] / 20.f;
                s[3] = ux;
                s[4] = uy;
                if (f.road_idx) f.road_idx[(size_t)a * kFullKR + slot] = k;
            }
            nr += __popc(bal);
        }
    }
    nr = min(nr, kFullKR);
    for (int i = kFullRoad0 + kFullPt * nr + lane; i < kFullVeh0; i += 32) o[i] = 0.f;
    if (f.road_idx)
        for (int t = nr + lane; t < kFullKR; t += 32) f.road_idx[(size_t)a * kFullKR + t] = -1;

    // ---- vehicle context (24 x 7)
    const int self = a - wd.x;
    unsigned long long key = kKeyInf;
    if (lane < wd.y && lane != self) {
        const int b = wd.x + lane;
        if (status_of(f.st.meta[b]) & kAlive) {
            const float4 pb = f.st.pos[b];
            const float dx = pb.x - p.x, dy = pb.y - p.y;
            key = key_of(dx * dx + dy * dy, lane);
        }
    }
    const int nv = min(__popc(__ballot_sync(kFull, key != kKeyInf)), kFullKV);
    key = warp_sort32(key, lane);
    if (lane < kFullKV) {
        float s[kFullNb] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        int jdx = -1;
        if (lane < nv) {
            const int b = wd.x + key_idx(key);
            const float4 pb = f.st.pos[b], qb = f.st.quat[b], vb = f.st.vel[b];
            float hjx, hjy, bx, by;
            heading_of(qb.x, qb.y, qb.z, qb.w, hjx, hjy);
            to_ego(hx, hy, pb.x - p.x, pb.y - p.y, bx, by);
            const float dpsi = atan2f(cross2(hx, hy, hjx, hjy), hx * hjx + hy * hjy);
            s[0] = bx / kSceneHalf;
            s[1] = by / kSceneHalf;
            s[2] = 2.f * kHalfLen / kSceneHalf;
            s[3] = 2.f * kHalfWid / kSceneHalf;
            s[4] = dpsi / 3.14159265358979323846f;
            s[5] = sqrtf(vb.x * vb.x + vb.y * vb.y) / 10.f;
            s[6] = ttc_pair(p.x, p.y, hx, hy, v.x, v.y, pb.x, pb.y, hjx, hjy, vb.x, vb.y) / kTtcMax;
            jdx = b;
        }
        float* r = o + kFullVeh0 + kFullNb * lane;
#pragma unroll
        for (int i = 0; i < kFullNb; ++i) r[i] = s[i];
        if (f.veh_idx) f.veh_idx[(size_t)a * kFullKV + lane] = jdx;
    }
    if (lane == 0) {
        if (f.n_road) f.n_road[a] = nr;
        if (f.n_veh) f.n_veh[a] = nv;
    }
}

cudaError_t sf_launch_full_obs(const FullObsArgs& f, cudaStream_t s) {
    if (f.num_agents <= 0) return cudaSuccess;
    constexpr int NW = 8;
    full_obs_kernel<NW><<<(f.num_agents + NW - 1) / NW, 32 * NW, 0, s>>>(f);
    return cudaGetLastError();
}
