// sf_internal.cuh -- device-side layouts and constants of the vehicle step.
//
// Constants follow SceneFactory (arXiv 2605.08528): actuation App. F
// Tab. app_action_params, rewards App. G Tab. app_reward_terms, observations
// App. D, scene rules App. C; the vehicle of the benchmark workload (1500 kg,
// 4.5 x 1.8 m box, r_w 0.33 m, k 35 kN/m, c 4 kN s/m, rest 0.3 m); where the
// paper is silent the value is a stated reading.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace sfk {

// ---------------------------------------------------------------- vehicle
constexpr double kMassD = 1500.0;
constexpr double kLenD = 4.5, kWidD = 1.8, kHgtD = 0.5;       // box; height is a reading
constexpr float kG = 9.81f;
constexpr float kMass = 1500.0f;
constexpr float kInvMass = (float)(1.0 / kMassD);
constexpr float kHalfLen = 2.25f, kHalfWid = 0.9f;
// uniform box inertia m/12 (b^2 + c^2) and its inverse
constexpr double kIxxD = kMassD / 12.0 * (kWidD * kWidD + kHgtD * kHgtD);
constexpr double kIyyD = kMassD / 12.0 * (kLenD * kLenD + kHgtD * kHgtD);
constexpr double kIzzD = kMassD / 12.0 * (kLenD * kLenD + kWidD * kWidD);
constexpr float kIxx = (float)kIxxD, kIyy = (float)kIyyD, kIzz = (float)kIzzD;
constexpr float kInvIxx = (float)(1.0 / kIxxD), kInvIyy = (float)(1.0 / kIyyD), kInvIzz = (float)(1.0 / kIzzD);
constexpr float kHardX = 1.3f, kHardY = 0.8f, kHardZ = -0.25f; // wheelbase 2.6 m (Sec. 3.2), track 1.6 m
constexpr float kWheelR = 0.33f;
constexpr float kKSusp = 35000.0f, kCSusp = 4000.0f, kRest = 0.3f;
constexpr double kWheelID = 0.5 * 37.5 * 0.33 * 0.33 * 1.094;  // m_wheel, s_inertia (App. F)
constexpr float kWheelI = (float)kWheelID;
constexpr float kInvWheelI = (float)(1.0 / kWheelID);
constexpr float kWheelR2OverI = (float)(0.33 * 0.33 / kWheelID);
constexpr float kSteerI = 1.0f;
constexpr float kThetaMax = 0.45f, kKp = 1839.5f, kKd = 110.5f, kTauSteer = 1200.0f;
constexpr float kTauDrive = 600.7f, kTauBrkF = 1090.5f, kTauBrkR = 980.7f;
constexpr float kLambdaYaw = 10.6f;
constexpr float kUzMin = 0.05f;
constexpr float kKContact = 1.0e6f, kCContact = 1.6e4f;
constexpr float kDampRamp = 0.01f;   // suspension / contact dampers ramp in over 1 cm
constexpr float kWheelbase = 2.6f;
// static equilibrium height: hardpoint depth + (rest - m g / 4k) + wheel radius
constexpr float kZStar = (float)(0.25 + (0.3 - kMassD * 9.81 / (4.0 * 35000.0)) + 0.33);
// bounding-circle cull of footprint pairs: 2 * sqrt(hl^2 + hw^2), squared
constexpr float kPairCull2 = (float)(4.0 * (2.25 * 2.25 + 0.9 * 0.9));
constexpr float kPairCullR = 4.8466483f;   // sqrt(kPairCull2), rounded up

// ---------------------------------------------------------------- kinematic bicycle backend (Sec. 4.4)
constexpr float kBikeThetaMax = 0.52359877559829887f;                          // 30 degrees
constexpr float kBikeADrive = (float)(2.0 * 600.7 / (0.33 * 1500.0));          // both front drive torques / (r m)
constexpr float kBikeABrake = (float)(2.0 * (1090.5 + 980.7) / (0.33 * 1500.0));  // all four brakes / (r m)

// ---------------------------------------------------------------- rewards / events (App. G)
constexpr float kGoalR = 3.0f, kWGoal = 45.0f, kWCollision = 6.0f, kWCrash = 10.0f, kWLaneForb = 20.0f;
constexpr float kWProgress = 2.0f, kProgressClip = 2.0f;
constexpr float kWLane = 0.08f, kLaneSigma = 1.75f, kLaneWh = 0.8f;
constexpr float kWOffroad = 0.5f, kOffroadLat = 3.25f, kOffroadDist = 6.0f;
constexpr float kWIdle = 0.05f, kIdleSpeed = 1.0f;
constexpr float kTtcAlphaV = 0.10f, kTtcPmaxV = 0.35f, kTtcFloor = 0.5f, kTtcMax = 10.0f;
constexpr float kTtcAlphaE = 0.07f, kTtcPmaxE = 0.40f, kEdgeHorizon = 40.0f;
constexpr float kDracThresh = 3.4f, kWDrac = 0.01f, kDracGapFloor = 0.1f;
constexpr float kDriftMax = 100.0f, kTiltGz = -0.15f;
constexpr int kWarmup = 24, kMaxSteps = 1500;
constexpr float kSceneHalf = 100.0f, kSegGapMax = 3.0f, kEdgeHalfWidth = 0.05f;
// three TTC circles (App. D): r = max(0.45, 0.55 W), d = min(WB/2, max(0, L/2 - 0.8 r))
constexpr float kCircR = 0.99f;
constexpr float kCircD = 1.3f;

// ---------------------------------------------------------------- resets
constexpr float kSpawnGoalMin = 50.0f, kSpawnGoalMax = 150.0f;
constexpr float kSpawnVMin = 5.0f, kSpawnVMax = 20.0f;
constexpr float kSpawnSpacing = 10.0f, kParkX = 1000.0f;
constexpr int kSpawnTries = 8;

// ---------------------------------------------------------------- road grid
constexpr double kCellMin = 4.0;   // grid cell edge [m]; larger when a world spans > 128 cells
constexpr int kGridMax = 128;
constexpr double kEdgeCellMin = 16.0;   // edge-grid cell edge [m]
constexpr int kEdgeGridMax = 16;
constexpr float kSegReach = 3.0f;  // no segment is longer (App. C gap rule)
constexpr float kKnnR0 = 10.0f, kLaneR0 = 6.0f, kGrow = 1.6f;
constexpr float kHintJump = 20.0f;   // a hint farther than this from the agent is not used

// ---------------------------------------------------------------- layout
constexpr int kMaxAgents = 32;
constexpr int kK = 8, kL = 32;
constexpr int kObsEgo = 16, kObsNbr = 10, kObsPt = 7;
constexpr int kObsDim = kObsEgo + kK * kObsNbr + kL * kObsPt;  // 320
// the paper's full observation (App. D): ego 11, 350 road slots x 5, 24 vehicle slots x 7
constexpr int kFullEgo = 11, kFullKR = 350, kFullPt = 5, kFullKV = 24, kFullNb = 7;
constexpr int kFullRoad0 = kFullEgo, kFullVeh0 = kFullEgo + kFullKR * kFullPt;
constexpr int kFullObs = kFullVeh0 + kFullKV * kFullNb;         // 1929
constexpr float kFullR2 = 100.0f;                               // road radius 10 m, squared

// point meta bits (input-order store)
constexpr uint32_t kPtTypeMask = 0xFFu;
constexpr uint32_t kPtSegNext = 1u << 8;   // point k and k+1 form a segment
constexpr uint32_t kPtLane = 1u << 9;      // Waymo type 1 or 2
constexpr uint32_t kPtEdge = 1u << 10;     // Waymo type 15 or 16
// info word of a cell-sorted record: input index within the world (bits 0-15),
// Waymo type (16-23) and these bits
constexpr uint32_t kInfoSegNext = 1u << 24;
constexpr uint32_t kInfoLane = 1u << 25;
constexpr uint32_t kInfoEdge = 1u << 26;
constexpr uint32_t kInfoHasNext = 1u << 27;  // the polyline continues after the point
constexpr int kMaxWorldPoints = 65535;       // a world's points are indexed by 16 bits
constexpr int kMaxStageBytes = 160 * 1024;   // dynamic shared memory of a staging block

// status and event bits (same values as the public header)
constexpr uint32_t kAlive = 1u, kParked = 2u;
constexpr uint32_t kEvGoal = 1u, kEvCollision = 2u, kEvCrash = 4u, kEvLaneForb = 8u, kEvOffroad = 16u,
                   kEvIdle = 32u, kEvTimeout = 64u, kEvNonfinite = 128u, kEvRespawned = 256u;
constexpr int kFlagInvincible = 1, kFlagAutoReset = 2, kFlagRecord = 4;
constexpr int kFlagWeatherAll = 1 << 16;   // internal: the ALL weather model (set from sf_config)

}  // namespace sfk

// Agent state, structure of float4 arrays, one element per agent.
struct DevState {
    float4* pos;     // px, py, pz, delta
    float4* quat;    // qw, qx, qy, qz
    float4* vel;     // vx, vy, vz, delta_dot
    float4* angv;    // wx, wy, wz, mu
    float4* spin;    // wheel spins FL FR RL RR
    float4* goal;    // gx, gy, start x, start y
    float* peak_drac;
    uint32_t* meta;  // precip | surface << 8 | status << 16
    int32_t* step;
    int32_t* episode;
};

// One world's road blob (built on the host at load time, 16-byte aligned
// sections, copied whole into shared memory by a block that stages it):
//   u16    coff[nx*ny + 1]  cell offsets into the records (relative to the world)
//   float4 seg[np]          the world's points sorted by grid cell, row-major,
//                           stable, as (x, y, x', y'): (x', y') the next point of
//                           the polyline, the previous one at its end, the
//                           point itself for a one-point polyline
//   u32    info[np]         input index within the world | type << 16 | kInfo*
//   float4 edge[ecnt]       the world's road-edge segments (a, b), sorted by the
//                           cell of a in a coarser edge grid (row-major, stable)
//   u16    eoff[ex*ey + 1]  edge-grid cell offsets into edge
// Cell (cx, cy) = floor((x - x0) / c), clamped; the cells of one grid row form
// one contiguous range [coff[cy*nx + cx0], coff[cy*nx + cx1 + 1]).  Segments
// are found through their start points.  The edge grid has the same origin
// and cells of ce >= kEdgeCellMin (at most kEdgeGridMax per side).
struct DevGrid {
    float x0, y0, c, inv_c;
    int nx, ny, np, ecnt;
    int bytes, o_seg, o_info, o_edge;   // blob size and section offsets [bytes]
    int q0, pad;                        // the world's first point (input order)
    unsigned long long blob;            // byte offset of the blob in the road store
    float inv_ce;                       // the edge grid: 1 / cell size, cells per side, offsets [bytes]
    int ex, ey, o_eoff;
};

// Road store of all worlds.
// Road answers at one spawn candidate (a lane point), computed once when the
// roads are loaded by the step's own exact queries: a respawned agent stands
// exactly on its candidate, so its nearest lane and 32 nearest road points
// are these, and no query runs at respawn time.
struct SpawnQ {
    uint16_t pos[32];            // sorted record positions of the 32 nearest points (0xFFFF: none)
    int seg;                     // nearest lane segment (input index), -1 none
    float dist, lat, tx, ty;     // its distance; lateral offset and tangent before the goal orientation
    float d32;                   // distance of the 32nd point (0: fewer than 32)
    int pad[2];
};
static_assert(sizeof(SpawnQ) == 96, "spawn table entry layout");

struct DevRoads {
    const int4* world;          // (first agent, agent count, first point, point count)
    const int2* cand;           // (first spawn candidate, candidate count)
    const float4* pt;           // (x, y, road direction x, y), input order
    const int32_t* pend;        // one past the last point of the point's polyline
    const float* arc;           // arc length from the polyline's first point (summed in double)
    const int32_t* cands;       // spawn candidate point indices
    const DevGrid* grid;        // per world
    const unsigned char* blob;  // every world's road blob
    const float4* mid;          // per point k: midpoint and unit direction of segment k -> k+1
                                // (App. C rule), x = +inf when k starts no segment
    const uint8_t* ptype;       // per point: Waymo type of its polyline
    int agent_base;             // index in the whole CSR of the first agent (world range)
    const SpawnQ* spawnq;       // per spawn candidate (indexed like cands), null: none built
};

struct DevOutputs {
    float* obs;
    float* reward;
    uint8_t* done;
    uint32_t* events;
    int32_t* lane_seg;
    int32_t* knn_pts;
    int32_t* knn_agents;
    float* drac;
    unsigned int* error_word;  // bit0 non-finite seen
    float* hint;               // [A][4] last query: 32nd-point distance, nearest-lane distance (0 = unknown)
                               // and the position (x, y) they were measured from
};

enum WorldMode { kModeStep = 0, kModeReset = 1, kModeObserve = 2 };

// results of one agent's road queries for the events
struct AgentQ {
    int seg;                     // nearest lane segment (input index), -1 none
    float dist, lat, tx, ty;     // its distance, signed lateral offset, tangent toward the goal
    float tedge;                 // edge-ray time (inf: no edge within 40 m)
    int forb, need;              // lane-forbidden; road block to recompute
};

// per-agent scratch of the split step (kernels exchange through it)
struct StepScratch {
    AgentQ* q;                   // [A] event queries
    float2* prev;                // [A] start-of-step position
    float2* head;                // [A] heading after the physics, then after respawns
    uint8_t* flag;               // [A] bit 0 non-finite this step, bit 1 road block stale
    const int32_t* agent_world;  // [A] world of each agent
    int32_t* fix_list;           // [A] agents whose road block is stale, in arrival order
    unsigned* fix_count;         // [1] their number (reset by the physics kernel)
};

struct WorldArgs {
    DevState st;
    DevRoads rd;
    DevOutputs out;
    const int4* packs;      // (first world, worlds, first agent, agents) per thread block
    int num_packs;
    int stage_bytes;        // shared memory per block for staged road blobs (0: read them from global)
    StepScratch sc;         // split step only
    const float* actions;   // [A][3]   (step mode)
    const uint8_t* mask;    // [A]      (reset mode)
    int num_worlds;
    int num_agents;
    int dynamics;           // 0 raycast vehicle (substeps), 1 kinematic bicycle (one update per step)
    float h;                // substep length
    int substeps;
    int flags;
    unsigned long long seed;
    // dynamics surrogate (optional): normalised MLP outputs [A][16] and the
    // output statistics (mean[16], std[16]); mode 0 off, 1 replace the substeps
    // of gated agents, 2 audit (physics runs, the surrogate's position error is
    // recorded as the max into *audit_err)
    const float* surr_y;
    const float* surr_stats;
    int surr_mode;
    unsigned int* audit_err;   // float bits, max-reduced
    unsigned int* surr_count;  // number of agents that used the surrogate (accumulated)
    // bounded wait of the road staging: limit in ns (0: 1 s); withhold != 0 sets
    // the barrier up but issues no copy (a test of the timeout path)
    unsigned long long wait_ns;
    int withhold;
    // optional: device views of page-locked host buffers [A] that also receive
    // the step's rewards and done flags (the host-buffer step, sf_step_host)
    float* host_reward;
    uint8_t* host_done;
};

// surrogate feature / target layout (dynamics surrogate of the step)
constexpr int kSurrIn = 30, kSurrInLd = 32, kSurrOut = 16;

// the full observation (App. D) of every agent from the current state
struct FullObsArgs {
    DevState st;
    DevRoads rd;
    const int32_t* agent_world;  // [A]
    int num_agents;
    float* obs;                  // [A][kFullObs]
    int32_t* n_road;             // [A] or null
    int32_t* n_veh;              // [A] or null
    int32_t* road_idx;           // [A][kFullKR] or null
    int32_t* veh_idx;            // [A][kFullKV] or null
    int weather_all;             // the weather byte is a water film (ALL model), not a precipitation class
};

// launch wrappers (sf_world.cu)
// the spawn table: one entry per spawn candidate c of rd.cands (its world cand_world[c])
cudaError_t sf_launch_spawn_table(const DevRoads& rd, const int32_t* cand_world, int ncand, SpawnQ* out,
                                  cudaStream_t s);
cudaError_t sf_launch_full_obs(const FullObsArgs& f, cudaStream_t s);
cudaError_t sf_launch_world(int mode, const WorldArgs& a, int warps_per_block, cudaStream_t s);
// one control step as four kernels (physics, road queries, events, fix-up); nwq warps per query block
cudaError_t sf_launch_step_split(const WorldArgs& a, int nwq, cudaStream_t s);
cudaError_t sf_launch_place(const WorldArgs& a, const float* d_place, cudaStream_t s);
// gate of the surrogate per agent (1 = eligible), from the current state
cudaError_t sf_launch_surr_gate(const WorldArgs& a, float dt, uint8_t* d_elig, cudaStream_t s);
// features [A][kSurrInLd] of the current state and actions; normalised when stats ([30] mean, [30] std) given
cudaError_t sf_launch_surr_features(const WorldArgs& a, const float* d_actions, const float* x_stats, float* d_x,
                                    cudaStream_t s);
// snapshot of the dynamic state (pos, quat, vel, angv, spin) into snap[5][A]
cudaError_t sf_launch_surr_snapshot(const WorldArgs& a, float4* snap, cudaStream_t s);
// targets of the step just taken from the snapshot; rows of gated, non-respawned agents are appended
// (features from d_x, targets) to out_x [cap][kSurrIn], out_y [cap][kSurrOut] at *count
cudaError_t sf_launch_surr_collect(const WorldArgs& a, const float4* snap, const uint8_t* d_elig, const float* d_x,
                                   float dt, float* out_x, float* out_y, unsigned long long cap,
                                   unsigned long long* count, cudaStream_t s);

// training kernels of the surrogate (sf_surrogate.cu)
cudaError_t sf_launch_col_stats(const float* x, unsigned long long n, int k, float* stats, cudaStream_t s);
cudaError_t sf_launch_gather(const float* x, const float* y, unsigned long long n, const float* xs, const float* ys,
                             int batch, unsigned long long seed, unsigned long long t, float* bx, float* by,
                             cudaStream_t s);
