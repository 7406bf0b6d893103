/*
 * sf.h -- C-ABI of the batched multi-world vehicle step on one B300 (sm_103a).
 *
 * The library steps many independent driving worlds at once, each holding up to
 * SF_MAX_AGENTS_PER_WORLD vehicles on its own z-flattened road map, following
 * SceneFactory (arXiv 2605.08528): 120 Hz physics under a 30 Hz control step
 * (Sec. 4.1), steering PD (Sec. 3.2, Eq. steer_pd), front-wheel drive and
 * four-wheel brakes (App. F, Tab. app_action_params), ego / neighbour / road
 * observations (App. D), ten reward terms and terminations (App. G,
 * Tab. app_reward_terms) and teleport-only resets (App. J).  The vehicle is a
 * raycast spring-damper chassis with friction-capped tire impulses integrated
 * by symplectic Euler over fixed substeps.
 *
 * Conventions
 *  - Every pointer named d_* is CUDA device memory owned by the caller; h_*
 *    pointers are host memory owned by the caller.  The library owns the agent
 *    state, the road store and its output buffers; none of them is exposed
 *    except through sf_output_ptrs.
 *  - Calls that launch work are asynchronous on the stream given to sf_create;
 *    caller buffers must stay valid until that stream reaches the call.
 *    Calls marked "synchronous" wait for the stream first.
 *  - Kernel-side conditions (non-finite states) are recorded in a device word
 *    and reported by the next synchronous call (sf_sync, sf_get_state, ...).
 *  - No call throws; every call returns an sf_status; sf_last_error gives the
 *    message of the last failure of a handle.  There is no CPU fallback: a
 *    missing or unusable GPU is SF_ERR_CUDA.
 */
#ifndef SF_H
#define SF_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sf_ctx* sf_handle;

typedef enum {
    SF_OK = 0,
    SF_ERR_INVALID_ARG = 1, /* bad pointer, size, CSR offsets or configuration         */
    SF_ERR_CUDA = 2,        /* a CUDA runtime call failed                               */
    SF_ERR_OOM = 3,         /* device allocation failed                                 */
    SF_ERR_NONFINITE = 4,   /* at least one agent state went non-finite since last sync */
    SF_ERR_TIMEOUT = 5,     /* a bounded device wait gave up                            */
    SF_ERR_STATE = 6        /* call order violated (e.g. sf_step before sf_load_roads)  */
} sf_status;

#define SF_MAX_AGENTS_PER_WORLD 32
#define SF_K_AGENTS 8   /* neighbours in the observation                   */
#define SF_L_POINTS 32  /* road points in the observation                  */
#define SF_OBS_EGO 16
#define SF_OBS_NBR 10
#define SF_OBS_PT 7
#define SF_OBS_DIM (SF_OBS_EGO + SF_K_AGENTS * SF_OBS_NBR + SF_L_POINTS * SF_OBS_PT) /* 320 */

/* Exchange layout of the agent state (sf_get_state / sf_set_state):
 * float columns (SF_NF per agent) */
enum {
    SF_F_PX = 0, SF_F_PY, SF_F_PZ,          /* CoM position [m], world frame, road plane z = 0 */
    SF_F_QW, SF_F_QX, SF_F_QY, SF_F_QZ,     /* attitude quaternion                              */
    SF_F_VX, SF_F_VY, SF_F_VZ,              /* CoM velocity [m/s]                               */
    SF_F_WX, SF_F_WY, SF_F_WZ,              /* angular velocity, world frame [rad/s]            */
    SF_F_S0, SF_F_S1, SF_F_S2, SF_F_S3,     /* wheel spin FL FR RL RR [rad/s]                   */
    SF_F_DELTA, SF_F_DDELTA,                /* front steering angle [rad] and rate [rad/s]      */
    SF_F_GX, SF_F_GY,                       /* goal [m]                                         */
    SF_F_SX, SF_F_SY,                       /* episode start [m]                                */
    SF_F_MU,                                /* tire-road friction coefficient                   */
    SF_F_PEAK_DRAC,                         /* episode peak DRAC [m/s^2]                        */
    SF_NF
};
/* int32 columns (SF_NI per agent) */
enum {
    SF_I_PRECIP = 0,  /* 0 dry, 1 light rain, 2 heavy rain, 3 snow        */
    SF_I_SURFACE,     /* 0 asphalt, 1 concrete, 2 gravel                  */
    SF_I_STEP,        /* control steps since spawn                        */
    SF_I_EPISODE,     /* episodes started by this agent slot              */
    SF_I_STATUS,      /* SF_STATUS_* bits                                 */
    SF_I_EVENTS,      /* SF_EV_* bits of the last step                    */
    SF_NI
};
#define SF_STATUS_ALIVE 1u
#define SF_STATUS_PARKED 2u

/* event bits written per agent per step (App. G) */
#define SF_EV_GOAL (1u << 0)
#define SF_EV_COLLISION (1u << 1)
#define SF_EV_CRASH (1u << 2)
#define SF_EV_LANE_FORBIDDEN (1u << 3)
#define SF_EV_OFFROAD (1u << 4)
#define SF_EV_IDLE (1u << 5)
#define SF_EV_TIMEOUT (1u << 6)
#define SF_EV_NONFINITE (1u << 7)
#define SF_EV_RESPAWNED (1u << 8)

/* sf_config.flags */
#define SF_FLAG_INVINCIBLE 1     /* events are logged but never terminate (Sec. 4.1)    */
#define SF_FLAG_AUTO_RESET 2     /* done agents respawn inside sf_step; else they park   */
#define SF_FLAG_RECORD_INDICES 4 /* keep nearest-lane and k-NN indices for inspection    */
#define SF_FLAG_METRICS 8        /* count ended episodes on the device (sf_get_metrics)  */

typedef struct {
    uint64_t seed;           /* seed of the counter-based reset draws                 */
    int32_t flags;           /* SF_FLAG_* bits                                        */
    int32_t warps_per_block; /* world-kernel launch shape; 0 = library default        */
    int32_t pack_agents;     /* 0: one world per thread block; 1..32: consecutive     *
                              * worlds share a block while their agents total at most *
                              * this many (worlds with more agents get a block alone) */
    int32_t stage_bytes;     /* shared memory per block (multiple of 16, at most      *
                              * 163840) into which a block copies its worlds' road    *
                              * data before querying it; 0 = query global memory.    *
                              * With staging, blocks also hold at most this many      *
                              * bytes of road data (a larger world is read from      *
                              * global memory)                                        */
    int32_t split_step;      /* 0: a step is one fused kernel; 1: four kernels        *
                              * (physics and events one warp per block of worlds,     *
                              * road queries one warp per agent, warps_per_block      *
                              * warps per query block); bit-identical results        */
    int32_t dynamics;        /* SF_DYN_VEHICLE (default): the raycast spring-damper   *
                              * vehicle over `substeps` substeps with footprint       *
                              * contact; SF_DYN_BICYCLE: the kinematic bicycle of the *
                              * paper's dynamics ablation (Sec. 4.4), one update per  *
                              * control step: steer 30 deg x a1, acceleration         *
                              * 2.43 m/s^2 x throttle - 8.37 m/s^2 x brake (the       *
                              * vehicle's actuator limits), no reversing, slip angle  *
                              * atan(tan(delta) / 2), no suspension, contact response *
                              * or lateral slip.  Events, rewards, observations and  *
                              * resets are the same for both                          */
    int32_t world_begin;     /* world range [world_begin, world_end) of the CSR given  */
    int32_t world_end;       /* to sf_load_roads that this handle steps (both 0: every *
                              * world).  Worlds are independent (no term of the step  *
                              * couples two worlds), so one handle per GPU over       *
                              * disjoint ranges shards a batch with no exchange; a    *
                              * shard's worlds evolve bit-identically to the same    *
                              * worlds in one handle over all of them (the respawn    *
                              * draws use the agent's index in the whole CSR).  Agent *
                              * indices of the handle's outputs are local to the      *
                              * range                                                 */
    int32_t weather_model;   /* SF_WEATHER_TABLE (default): mu from the (precip,       *
                              * surface) table; SF_WEATHER_ALL: the modified ALL     *
                              * weather-to-friction model of Sec. 3.3 / App. B:      *
                              * surface 0 AC, 1 SMA, 2 OGFC and a water film h per   *
                              * agent (sf_roads.film_mm), mu = the model's static    *
                              * friction at 13.89 m/s (the printed curve points      *
                              * joined linearly, falling to the 1e-3 floor at the    *
                              * 0.85 mm aquaplaning threshold), and the ego group's  *
                              * weather token = Eq. weather_obs (h / 1 mm, one-hot   *
                              * AC, SMA, OGFC).  The film is resolved to 0.01 mm and *
                              * held to at most 2.55 mm (beyond 0.85 mm mu is the    *
                              * floor anyway)                                         */
    int32_t reserved[1];     /* must be zero                                          */
} sf_config;
#define SF_DYN_VEHICLE 0
#define SF_DYN_BICYCLE 1
#define SF_WEATHER_TABLE 0
#define SF_WEATHER_ALL 1

/* Worlds as CSR (host memory, read during sf_load_roads only).
 * World w holds agents [agent_off[w], agent_off[w+1]) (at most 32) and
 * polylines [poly_off[w], poly_off[w+1]); polyline p holds points
 * [point_off[p], point_off[p+1]) with Waymo type poly_type[p]
 * (1, 2 driving lanes; 15, 16 road edges; others are map points only).
 * Coordinates are world-local metres (each world centred at its origin,
 * App. C).  precip/surface give each agent's weather cell of the friction
 * table. */
typedef struct {
    int32_t num_worlds;
    int32_t num_polylines;
    int32_t num_points;
    const int32_t* agent_off;  /* [num_worlds + 1], agent_off[0] == 0, nondecreasing   */
    const int32_t* poly_off;   /* [num_worlds + 1], poly_off[0] == 0, nondecreasing    */
    const int32_t* point_off;  /* [num_polylines + 1], point_off[0] == 0, nondecreasing */
    const uint8_t* poly_type;  /* [num_polylines]                                       */
    const float* px;           /* [num_points]                                          */
    const float* py;           /* [num_points]                                          */
    const uint8_t* precip;     /* [num_agents] 0..3 (table weather model)               */
    const uint8_t* surface;    /* [num_agents] 0..2                                     */
    const float* film_mm;      /* [num_agents] water film [mm], finite and >= 0; read   *
                                * only with SF_WEATHER_ALL (precip is then ignored)    */
} sf_roads;

/* Device pointers to the library-owned outputs of the last sf_step / sf_reset.
 * Valid until sf_destroy or the next sf_load_roads. */
typedef struct {
    float* obs;            /* [A][SF_OBS_DIM] float32                          */
    float* reward;         /* [A]                                              */
    uint8_t* done;         /* [A] 1 if the agent terminated or timed out       */
    uint32_t* events;      /* [A] SF_EV_* bits                                 */
    int32_t* lane_seg;     /* [A] nearest lane segment start point, -1 if none (SF_FLAG_RECORD_INDICES) */
    int32_t* knn_points;   /* [A][SF_L_POINTS] global point indices, -1 pad     (SF_FLAG_RECORD_INDICES) */
    int32_t* knn_agents;   /* [A][SF_K_AGENTS] global agent indices, -1 pad     (SF_FLAG_RECORD_INDICES) */
    float* drac;           /* [A] DRAC of the last step                        */
    int32_t num_agents;
} sf_outputs;

/* Create a context on the current CUDA device: the batch of worlds and agents
 * that SceneFactory exposes as GPU-resident tensors of shape (num_envs,
 * num_agents, d) (Sec. 1; App. K "Batched joint-state tensors"), here owned
 * by the library and stepped by its kernels.  cuda_stream is a cudaStream_t
 * (NULL = legacy default stream) on which every call of this handle enqueues
 * its work.  *out receives the handle.  cfg may be NULL (all defaults).
 * Errors: SF_ERR_INVALID_ARG (NULL out, nonzero reserved, pack_agents outside
 * 0..32, bad stage_bytes, split_step, dynamics or world range), SF_ERR_CUDA
 * (no usable device). */
sf_status sf_create(const sf_config* cfg, void* cuda_stream, sf_handle* out);

/* Release every device and host resource of h (synchronous).  NULL is a no-op. */
sf_status sf_destroy(sf_handle h);

/* Validate the CSR on the host (offsets monotone and in range, at most 32
 * agents per world, finite coordinates, known weather codes), upload it, build
 * the derived road store (per-point road direction, App. C segment rule: gaps
 * > 3 m and endpoints outside the 200 m box are not segments; spawn candidates)
 * and allocate the agent state, every agent inactive.  Synchronous.  Replaces
 * any previous roads and state.  Errors: SF_ERR_INVALID_ARG, SF_ERR_OOM. */
sf_status sf_load_roads(sf_handle h, const sf_roads* h_roads);

/* One control step of every world (Sec. 4.1; App. F-G): `substeps` physics
 * substeps of dt/substeps each with the actions held, footprint contact
 * between the agents of a world at every substep, then events, rewards and
 * done flags, done agents parked or (SF_FLAG_AUTO_RESET) respawned, then the
 * observations of every agent.  d_actions is [A][3] float32 (throttle, steer,
 * brake) in [-1, 1]; throttle and brake are rectified, steer scales the
 * maximum steering angle (App. F).  Asynchronous.
 * Errors: SF_ERR_STATE (no roads), SF_ERR_INVALID_ARG (NULL actions, dt <= 0,
 * substeps outside 1..64), SF_ERR_CUDA (launch failure). */
sf_status sf_step(sf_handle h, const float* d_actions, float dt, int substeps);

/* The same control step end to end from host memory: h_actions [A][3] float32
 * is copied to the device, the step runs, and the rewards [A] float32 and done
 * flags [A] uint8 are copied into h_reward and h_done; returns when they are in
 * host memory (synchronous).  With a non-default stream and page-locked buffers
 * (cudaHostAlloc / cudaHostRegister) the transfers and the step are captured
 * into one CUDA graph that later calls with the same dt and substeps replay
 * (other page-locked buffers retarget its transfers); buffers with a device
 * mapping are read and written in place by the step's own kernels (the actions
 * loaded, rewards and done flags stored over the host link, also into the
 * device outputs), others by copy nodes.  The graph is re-captured after sf_load_roads or
 * sf_autotune.  Pageable buffers or the legacy stream run copies and the step
 * without a graph.  The buffers are caller-owned and must stay valid during the
 * call.
 * Errors: SF_ERR_STATE (no roads), SF_ERR_INVALID_ARG (NULL buffer, dt <= 0,
 * substeps outside 1..64), SF_ERR_OOM, SF_ERR_CUDA. */
sf_status sf_step_host(sf_handle h, const float* h_actions, float* h_reward, uint8_t* h_done, float dt,
                       int substeps);

/* sf_step_host for a host that consumes the observations too: the same call,
 * plus the step's observations [A][SF_OBS_DIM] float32 (1,280 B per agent)
 * copied into h_obs by the copy engine inside the same graph (a copy node;
 * page-locked h_obs required for the graph, else plain copies).  Switching
 * between sf_step_host and this call re-captures the graph.
 * Errors: as sf_step_host; SF_ERR_INVALID_ARG if h_obs is NULL. */
sf_status sf_step_host_obs(sf_handle h, const float* h_actions, float* h_obs, float* h_reward, uint8_t* h_done,
                           float dt, int substeps);

/* Autotuner: time each launch shape of the step over `iters` steps with the
 * given actions and keep the fastest for this handle.  Shapes s < 32 are the
 * fused kernel with 1 << (s & 3) warps per block, world packing when bit 2 is
 * set (blocks of at most pack_agents agents, 32 when the handle was created
 * with 0) and road staging budget (s >> 3) of {0, 49152, 98304, the handle's
 * stage_bytes when it is none of these} bytes; shapes 32 + k (k < 6) are the
 * split step with 2 << (k % 3) warps per query block, packed when k >= 3.  The agent state and every output are saved
 * before and restored after the trials, so the call does not advance the
 * simulation.  Synchronous; uses a temporary device buffer the size of the
 * state and outputs.  out_shape (may be NULL, [4]) receives the chosen warps
 * per block, pack_agents (0 = no packing), stage_bytes and split_step; out_ms
 * (may be NULL, [SF_AUTOTUNE_SHAPES]) the mean step time of each shape in ms
 * (0 for shapes not tried).
 * Errors: SF_ERR_STATE (no roads), SF_ERR_INVALID_ARG (iters < 1), SF_ERR_OOM. */
#define SF_AUTOTUNE_SHAPES 38
sf_status sf_autotune(sf_handle h, const float* d_actions, float dt, int substeps, int iters, int32_t* out_shape,
                      float* out_ms);

/* Copy the observations, rewards, done flags and event bits of the last step
 * or reset into caller device buffers ([A][SF_OBS_DIM], [A], [A], [A]); any
 * pointer may be NULL.  Asynchronous device-to-device copies.  The
 * observation is this library's 320-value analogue of App. D (ego 16 with
 * the weather token of Eq. weather_obs, 8 nearest agents x 10 with the
 * swept-circle TTC, 32 nearest road points x 7); rewards are the ten terms of
 * App. G (Tab. app_reward_terms) plus DRAC; done marks the sparse events and
 * the 1,500-step time-out (App. G "Termination and time-out"). */
sf_status sf_get_obs(sf_handle h, float* d_obs, float* d_reward, uint8_t* d_done, uint32_t* d_events);

/* Copy the inspection outputs of the last step / reset into caller device
 * buffers: nearest lane segment [A], k nearest road points [A][SF_L_POINTS],
 * k nearest agents [A][SF_K_AGENTS] (all int32, -1 = none; only maintained
 * with SF_FLAG_RECORD_INDICES) and the step DRAC [A] float32 (App. G reading:
 * max over the k nearest agents of closing speed^2 / (2 gap)).  Any pointer
 * may be NULL.  Asynchronous device-to-device copies. */
sf_status sf_get_indices(sf_handle h, int32_t* d_lane_seg, int32_t* d_knn_points, int32_t* d_knn_agents,
                         float* d_drac);

/* Episode metrics of Sec. 4 (the paragraph that defines SR, CR and DRAC),
 * over the episodes that ended since the handle was loaded or the counters
 * were last cleared.  With SF_FLAG_METRICS every step (sf_step, the captured
 * graphs, sf_step_host, the surrogate step) is followed by a small kernel that
 * keeps, per agent, the running episode's maximum step DRAC (the value of
 * sf_get_indices) and the union of its event bits, and adds each episode that
 * ends (done) to the counters: the success rate is the share of ended
 * episodes that reached their goal, the collision rate the share with an
 * inter-vehicle contact (the collision event, App. G; depth > 0 stands for
 * the paper's 25 N contact threshold), and the DRAC figure the mean over
 * ended episodes of their maximum DRAC, with the share above the paper's
 * 3.4 m/s^2 highway threshold.  A masked reset (sf_reset) starts new episodes
 * of the masked agents without counting the interrupted ones.  Counters are
 * integers (the DRAC sum in units of 1e-6 m/s^2, each episode's maximum held
 * to 1e6), so they do not depend on the order of the agents. */
typedef struct {
    uint64_t episodes;        /* ended episodes; the others count those in which the */
    uint64_t goals;           /* event (SF_EV_*) occurred at some step: goal reached */
    uint64_t collisions;      /* inter-vehicle contact                               */
    uint64_t crashes;         /* below the ground, drifted or tipped over            */
    uint64_t offroad;         /* off the road                                        */
    uint64_t lane_forbidden;  /* in a forbidden lane                                 */
    uint64_t idle;            /* idle                                                */
    uint64_t timeouts;        /* the time-out                                        */
    uint64_t nonfinite;       /* a non-finite state                                  */
    uint64_t drac_over;       /* ended episodes whose maximum DRAC exceeded 3.4 m/s^2 */
    double success_rate;      /* goals / episodes (SR), 0 without an ended episode   */
    double collision_rate;    /* collisions / episodes (CR)                          */
    double mean_episode_max_drac;  /* m/s^2                                          */
    double drac_over_rate;    /* drac_over / episodes                                */
} sf_metrics;

/* The counters into *out (synchronises the handle's stream).
 * Errors: SF_ERR_INVALID_ARG (NULL), SF_ERR_STATE (no roads, or the handle was
 * created without SF_FLAG_METRICS), SF_ERR_CUDA. */
sf_status sf_get_metrics(sf_handle h, sf_metrics* out);
/* Clears the counters (asynchronous on the handle's stream); episodes under
 * way count when they end.  Errors: as sf_get_metrics. */
sf_status sf_reset_metrics(sf_handle h);

/* The paper's full observation (SceneFactory App. D), 1,929 values per agent,
 * computed from the current state (after any sf_step / sf_reset / placement):
 *   [0, 11)       ego: goal in the body frame / 100 (x, y), sin and cos of the
 *                 goal bearing, goal distance / 100, body-frame velocity / 10
 *                 (x, y), then the weather token of Eq. weather_obs in this
 *                 library's weather cells: precip / 3, one-hot asphalt,
 *                 concrete, gravel;
 *   [11, 1761)    road context, 350 slots x 5: the midpoints of the world's
 *                 road segments (App. C: consecutive points of a polyline at
 *                 most 3 m apart, both inside the 200 m box) within 10 m of the
 *                 agent's centre, in ascending segment index (polyline order,
 *                 then point order), the first 350; per slot the body-frame
 *                 offset / 10 (x, y), polyline type / 20 and the body-frame
 *                 unit direction (x, y);
 *   [1761, 1929)  vehicle context, 24 slots x 7: the 24 nearest alive other
 *                 agents of the world (squared distance, ties to the lower
 *                 index); per slot the body-frame offset / 100 (x, y), length
 *                 / 100, width / 100, relative heading / pi, speed / 10 and the
 *                 swept three-circle time to collision / 10.
 * Slots beyond the filled ones are zero, and a parked agent's row is all zeros.
 * d_obs [A][SF_FULL_OBS_DIM] float32 (required); d_n_road, d_n_veh [A] int32
 * receive the number of filled road / vehicle slots (the slots are a prefix;
 * these counts are the masks of the policy's max-pool); d_road_idx
 * [A][SF_FULL_KR] and d_veh_idx [A][SF_FULL_KV] int32 receive the global
 * start-point index of each selected segment and the global index of each
 * selected agent, -1 past the end.  The optional pointers may be NULL.  All
 * buffers are caller-owned device memory.  Asynchronous on the handle's stream.
 * Errors: SF_ERR_STATE (no roads), SF_ERR_INVALID_ARG (NULL d_obs),
 * SF_ERR_CUDA. */
#define SF_FULL_EGO 11
#define SF_FULL_KR 350
#define SF_FULL_PT 5
#define SF_FULL_KV 24
#define SF_FULL_NB 7
#define SF_FULL_OBS_DIM (SF_FULL_EGO + SF_FULL_KR * SF_FULL_PT + SF_FULL_KV * SF_FULL_NB) /* 1929 */
sf_status sf_observe_full(sf_handle h, float* d_obs, int32_t* d_n_road, int32_t* d_n_veh, int32_t* d_road_idx,
                          int32_t* d_veh_idx);

/* Device pointers of the library-owned outputs (zero-copy). */
sf_status sf_output_ptrs(sf_handle h, sf_outputs* out);

/* Teleport-only reset (App. J): every agent with d_mask[a] != 0 starts a new
 * episode at a lane point drawn by a counter-based SplitMix64 hash of
 * (seed, agent, episode, attempt) with at least 50 m of lane ahead, heading
 * along the lane, goal 50-150 m ahead on the same lane, speed U[5, 20] m/s,
 * wheels rolling, at static equilibrium height, at least 10 m from the other
 * agents of its world when one of 8 attempts allows it (agents are processed
 * in index order).  Then the observations of every agent of every world that
 * had a masked agent are recomputed.  d_mask is [A] uint8.  Asynchronous. */
sf_status sf_reset(sf_handle h, const uint8_t* d_mask);

/* Place every agent explicitly: h_place is [A][6] = (x, y, heading, speed,
 * goal_x, goal_y); the agent starts an episode there at static equilibrium
 * height with rolling wheels.  Then all observations are computed.
 * Synchronous (host upload). */
sf_status sf_place_agents(sf_handle h, const float* h_place);

/* Read / write the whole agent state in the exchange layout: h_f is
 * [A][SF_NF] float32, h_i is [A][SF_NI] int32.  Synchronous.  sf_set_state
 * recomputes all observations.  sf_get_state reports a pending
 * SF_ERR_NONFINITE after copying. */
sf_status sf_get_state(sf_handle h, float* h_f, int32_t* h_i);
sf_status sf_set_state(sf_handle h, const float* h_f, const int32_t* h_i);

/* Checkpoint / resume the agent state to / from a file (little-endian header
 * + exchange layout).  Synchronous.  The roads must match (agent count). */
sf_status sf_save_state(sf_handle h, const char* path);
sf_status sf_load_state(sf_handle h, const char* path);

/* Wait for the handle's stream; return SF_ERR_NONFINITE / SF_ERR_TIMEOUT if the
 * device recorded such a condition since the last sync (and clear it). */
sf_status sf_sync(sf_handle h);

/* Failure detection of bounded device waits (no counterpart in the paper).
 * The step kernels wait on an mbarrier for the bulk copy that stages a
 * block's road blobs in shared memory; that wait gives up after limit_ns of
 * wall time (1 s by default; 0 gives up at the first poll), records a timeout
 * in the handle's device error word and carries on reading the roads from
 * global memory (same results); before the block exits it waits again,
 * bounded by 1 s whatever limit_ns is, for a copy it issued, so no copy
 * outlives the block.  The next synchronising call returns SF_ERR_TIMEOUT.
 * withhold_producer != 0 is for tests of that path: the barrier is set up
 * but no copy is issued, so the wait runs out on a barrier that nothing
 * completes, with no copy in flight.  Applies to later launches; a captured
 * graph keeps the values it was captured with.  SF_ERR_INVALID_ARG if h is
 * NULL. */
sf_status sf_set_wait_limit(sf_handle h, unsigned long long limit_ns, int withhold_producer);

/* ------------------------------------------------------------------------
 * BF16 tensor-core MLPs (dynamics surrogate and policy of the step).
 * An MLP of L dense layers y = act(W x + b), W [out, in] fp32 masters with
 * bf16 copies for the tcgen05 GEMMs, fp32 accumulation.  Hidden layers use
 * hidden_act, the last layer out_act (SF_ACT_*).  All device work runs on
 * the stream given to sf_mlp_create (or, for a step that uses the MLP, on the
 * world handle's stream).  An MLP keeps its activations in buffers of its
 * own: work that uses one MLP (or one surrogate) must not overlap on two
 * streams.
 * ---------------------------------------------------------------------- */
typedef struct sf_mlp* sf_mlp_handle;
#define SF_ACT_NONE 0
#define SF_ACT_ELU 1   /* the paper's network activation (App. E) */
#define SF_ACT_SILU 2
#define SF_ACT_TANH 3

/* dims[0..num_layers] are the layer widths (1..4096); 1 <= num_layers <= 8.
 * Weights start at zero.  Errors: SF_ERR_INVALID_ARG, SF_ERR_OOM, SF_ERR_CUDA. */
sf_status sf_mlp_create(int num_layers, const int32_t* dims, int hidden_act, int out_act, void* cuda_stream,
                        sf_mlp_handle* out);
sf_status sf_mlp_destroy(sf_mlp_handle m);
const char* sf_mlp_last_error(sf_mlp_handle m);

/* Set / read layer `layer`: h_w [out][in] and h_b [out] fp32 host arrays
 * (synchronous); sf_mlp_get_layer also returns the last gradients h_gw, h_gb
 * (any pointer may be NULL). */
sf_status sf_mlp_set_layer(sf_mlp_handle m, int layer, const float* h_w, const float* h_b);
sf_status sf_mlp_get_layer(sf_mlp_handle m, int layer, float* h_w, float* h_b, float* h_gw, float* h_gb);

/* Inference: d_y[b][0..out) = MLP(d_x[b][0..in)) for b < batch; d_x has row
 * stride ldx >= in floats, d_y row stride ldy >= out.  Asynchronous. */
sf_status sf_mlp_forward(sf_mlp_handle m, const float* d_x, int ldx, int batch, float* d_y, int ldy);

/* One training step on a batch (batch % 8 == 0): forward, mean-squared-error
 * loss against d_t [batch][out], backward through every layer (gradients kept
 * for sf_mlp_get_layer) and, if update != 0, an Adam step (beta 0.9, 0.999,
 * eps 1e-8) with learning rate lr.  h_loss (may be NULL) receives the loss
 * (synchronous when given). */
sf_status sf_mlp_train_step(sf_mlp_handle m, const float* d_x, const float* d_t, int batch, float lr, int update,
                            float* h_loss);

/* Inference without allocation, for callers that must not allocate device
 * memory once they run: code inside a captured or replayed CUDA graph whose
 * memory is fixed, callers under a device-memory budget that is already
 * spent, or hosts whose allocator is owned by someone else (the allocating
 * sf_mlp_forward grows its batch buffers with cudaMalloc on first use of a
 * larger batch).  The paper has no counterpart; this is a library service.
 *
 * Same result as sf_mlp_forward, but the bf16 layer inputs and the fp32
 * output live in one fixed 4 MiB device array compiled into this library
 * (sf_mlp_static_scratch_bytes() returns the size), so the call performs no
 * cudaMalloc, cudaFree or other allocation.  The array occupies 4 MiB on
 * every GPU that loads the library until the process exits.  A batch needs
 * batch * (2 * sum of the padded input widths of the layers + 4 * padded
 * output width) bytes (each part rounded up to 256 B); larger batches are
 * rejected with SF_ERR_INVALID_ARG and a message giving both sizes.  The
 * first call on a device looks the array's address up (cudaGetSymbolAddress)
 * and must therefore come before any stream capture on that device; a call
 * with batch 0 does only that lookup (d_x and d_y must still be non-NULL but
 * are not read or written), so a caller can prime the device before it has
 * real buffers.  Every
 * call clears and reuses the same array: calls that overlap on the GPU (on
 * different streams, or from different MLP handles) race and corrupt each
 * other's results; serialise them.  Asynchronous on the MLP's stream. */
sf_status sf_mlp_forward_static(sf_mlp_handle m, const float* d_x, int ldx, int batch, float* d_y, int ldy);
size_t sf_mlp_static_scratch_bytes(void);

/* Wait for the MLP's stream; SF_ERR_TIMEOUT if a GEMM's bounded wait gave up. */
sf_status sf_mlp_sync(sf_mlp_handle m);

/* The same for the MLP's tensor-core GEMMs (no counterpart in the paper):
 * their operand-ring mbarrier waits give up after limit_ns (1 s by default;
 * 0 gives up at the first poll), record SF_ERR_TIMEOUT for sf_mlp_sync and
 * skip the epilogue (the outputs of that launch are left unwritten); every
 * MMA and TMA load already issued is waited for (bounded by 1 s) before the
 * CTA frees its tensor memory and exits.  withhold_producer != 0 issues no
 * TMA load at all, so the first wait runs out with nothing in flight (tests
 * of that path).  SF_ERR_INVALID_ARG if m is NULL. */
sf_status sf_mlp_set_wait_limit(sf_mlp_handle m, unsigned long long limit_ns, int withhold_producer);

/* The GEMM itself: C = act(A . B^T + bias) with A [M][K], B [N][K] bf16
 * row-major device arrays (K % 8 == 0, 16-byte aligned), bias [N] or NULL,
 * outputs (any may be NULL): f32 [M][ldc], bf16 [M][ldc], transposed bf16
 * [N][ldt].  tile_n: 64, 128 or 256 output columns per CTA.  d_err (may be
 * NULL) is a device word that receives bit 2 if a bounded wait expired.
 * Asynchronous on cuda_stream. */
sf_status sf_gemm_bf16(const void* d_a, const void* d_b, const float* d_bias, int M, int N, int K, int act,
                       float* d_out_f32, void* d_out_bf16, void* d_out_bf16_t, int ldc, int ldt, int tile_n,
                       unsigned* d_err, void* cuda_stream);

/* ------------------------------------------------------------------------
 * Policy in the loop and the captured step graph.
 * ---------------------------------------------------------------------- */
/* One control step with actions from a policy MLP (320 inputs, 3 outputs,
 * e.g. 320->512->512->3 with tanh outputs): the policy reads the library's
 * current observations, writes a library-owned [A][3] action buffer, and the
 * step runs on them (the paper's loop of Alg. 1: observe, act, simulate).
 * Both run on the handle's stream.  Asynchronous. */
sf_status sf_step_policy(sf_handle h, sf_mlp_handle policy, float dt, int substeps);

/* The device's FP32 fused multiply-add throughput, measured: `iters` rounds of
 * eight independent FMA chains per thread, eight 256-thread blocks per SM, one
 * timed launch after a warm-up on `stream` (a cudaStream_t, NULL: the legacy
 * stream); *out_tflops = 2 x FMAs / elapsed time / 1e12.  The denominator of
 * the step's ALU roofline.  Synchronous.  Errors: SF_ERR_INVALID_ARG (NULL
 * out_tflops, iters < 1), SF_ERR_OOM, SF_ERR_CUDA. */
sf_status sf_fp32_fma_peak(void* stream, int iters, double* out_tflops);

/* Capture a whole control step into a CUDA graph on the handle's stream
 * (which must not be the legacy default stream): [policy forward if policy
 * != NULL] -> [surrogate features and MLP if surrogate != NULL] -> the step
 * (sf_step_surrogate with a surrogate, else sf_step; actions from the policy,
 * else from d_actions, whose contents may change between launches) ->
 * [sf_reset(d_reset_mask) if not NULL].  Buffers are allocated before the
 * capture.  Replays with sf_graph_launch run every kernel of the step with
 * one launch call; the handle's state evolves as with the individual calls.
 * Errors: SF_ERR_STATE, SF_ERR_INVALID_ARG, SF_ERR_OOM, SF_ERR_CUDA. */
typedef struct sf_graph* sf_graph_handle;
typedef struct sf_surrogate* sf_surrogate_handle;
sf_status sf_graph_capture(sf_handle h, sf_mlp_handle policy, sf_surrogate_handle surrogate, const float* d_actions,
                           const uint8_t* d_reset_mask, float dt, int substeps, sf_graph_handle* out);
sf_status sf_graph_launch(sf_graph_handle g);
sf_status sf_graph_destroy(sf_graph_handle g);

/* ------------------------------------------------------------------------
 * Learned dynamics surrogate: a BF16 MLP 30 -> 256 -> 256 -> 256 -> 16
 * (SiLU) that predicts one control step of the chassis of an agent that is
 * alone (no other footprint within 4.85 m + 2 m + |dv| dt), on mu >= 0.3, at
 * most 35 m/s and tilted less than 10 degrees; the physics substeps remain the
 * fallback for every other agent, and steering keeps its exact PD recurrence.
 * Inputs (30, heading frame at t): z, tilt quaternion (4), v (3), omega (3),
 * wheel spins (4), suspension compressions (4) and rates (4), steer angle and
 * rate, decoded action (3), mu, 0.  Outputs (16): the step's change of
 * heading-frame position, body rotation vector, heading-frame velocity and
 * angular velocity (each minus the constant-velocity prediction) and of the
 * wheel spins, normalised by the training set's mean and deviation.
 * ---------------------------------------------------------------------- */

/* An untrained surrogate (seeded initial weights) on cuda_stream. */
sf_status sf_surrogate_create(void* cuda_stream, sf_surrogate_handle* out);
sf_status sf_surrogate_destroy(sf_surrogate_handle s);

/* One plain physics step of h with d_actions, recording a training
 * transition for every gated agent that stayed alive and neither respawned,
 * collided nor crashed: raw inputs appended to d_x [cap][30], raw outputs to
 * d_y [cap][16] at the device counter *d_count (advanced by the number of
 * transitions; rows beyond cap are dropped).  The rows of one call follow the
 * agents' order, so a seeded collection yields the same rows on every run.
 * Asynchronous on h's stream. */
sf_status sf_surrogate_collect(sf_handle h, sf_surrogate_handle s, const float* d_actions, float dt, int substeps,
                               float* d_x, float* d_y, unsigned long long cap, unsigned long long* d_count);

/* Fit the normalisation to the n collected rows and run `steps` Adam steps
 * (mean-squared error of the normalised outputs, batch rows drawn by a
 * counter hash of (seed, step, row), cosine-decayed learning rate from lr).
 * Synchronous; *h_loss (may be NULL) receives the last step's loss. */
sf_status sf_surrogate_train(sf_surrogate_handle s, const float* d_x, const float* d_y, unsigned long long n,
                             int batch, int steps, float lr, unsigned long long seed, float* h_loss);

/* The surrogate's MLP (for its weights) and its normalisation statistics
 * (host [92] = input mean[30], input std[30], output mean[16], output std[16]). */
sf_mlp_handle sf_surrogate_mlp(sf_surrogate_handle s);
sf_status sf_surrogate_stats(sf_surrogate_handle s, float* h_stats);
sf_status sf_surrogate_set_stats(sf_surrogate_handle s, const float* h_stats);

/* One control step with the surrogate: every gated agent's chassis follows the
 * MLP's prediction instead of the substep loop.  With audit != 0 every agent
 * runs the physics instead and the largest distance between the surrogate's
 * and the physics' end position over gated agents is recorded (the periodic
 * audit).  Asynchronous.  SF_ERR_STATE on a handle with SF_DYN_BICYCLE dynamics
 * (the surrogate stands in for the raycast vehicle only; so does
 * sf_surrogate_collect). */
sf_status sf_step_surrogate(sf_handle h, sf_surrogate_handle s, const float* d_actions, float dt, int substeps,
                            int audit);

/* Synchronous: the largest audit error since the last call [m] and the number
 * of agent-steps that used the surrogate; both counters are reset. */
sf_status sf_surrogate_audit(sf_handle h, float* h_max_err, unsigned long long* h_used);

/* ------------------------------------------------------------------------
 * The paper's late-fusion actor-critic network (SceneFactory App. E) on the
 * full observation (sf_observe_full).  Two networks without shared weights,
 * the actor and the critic, each:
 *   ego encoder      11 -> 64 -> 64 (ELU) on observation values [0, 11)
 *   road encoder     5 -> 96 -> 96 (ELU) on each road slot, then a masked
 *                    max-pool over the first n_road slots
 *   vehicle encoder  7 -> 96 -> 96 (ELU) on each vehicle slot, masked
 *                    max-pool over the first n_veh slots
 *   trunk            [ego | road | vehicles] 256 -> 128 -> 64 (ELU)
 *   head             actor: 3 action means; critic: 1 value (linear)
 * The masked max-pool is the paper's "fill padding with -inf, then max"; a
 * group without a filled slot pools to zeros.  Weights and activations are
 * bf16 on the tensor cores with fp32 accumulation; biases are fp32.
 * Parameters (fp32, host) are one flat vector: for the actor then the critic,
 * for each layer in the order ego0, ego1, road0, road1, veh0, veh1, trunk0,
 * trunk1, head, the weight [out][in] row-major then the bias [out]; then the
 * 3 log standard deviations of the diagonal Gaussian policy (kept, not used by
 * the forward pass).  sf_lf_num_params() gives the length.
 * ---------------------------------------------------------------------- */
typedef struct sf_lf* sf_lf_handle;

size_t sf_lf_num_params(void);

/* A network with all parameters zero on cuda_stream (NULL = legacy default
 * stream).  Errors: SF_ERR_INVALID_ARG (NULL out), SF_ERR_CUDA. */
sf_status sf_lf_create(void* cuda_stream, sf_lf_handle* out);
sf_status sf_lf_destroy(sf_lf_handle m);
const char* sf_lf_last_error(sf_lf_handle m);

/* Set / read every parameter (h_params has n == sf_lf_num_params() floats;
 * set rejects non-finite values).  Synchronous.  Errors: SF_ERR_INVALID_ARG. */
sf_status sf_lf_set_params(sf_lf_handle m, const float* h_params, size_t n);
sf_status sf_lf_get_params(sf_lf_handle m, float* h_params, size_t n);

/* Forward pass of both networks on num_agents observation rows:
 * d_obs [num_agents][SF_FULL_OBS_DIM] float32, d_n_road / d_n_veh [num_agents]
 * int32 filled-slot counts (clamped to 0..350 / 0..24), all as written by
 * sf_observe_full; d_mean [num_agents][3] receives the actor's action means,
 * d_value [num_agents] (may be NULL) the critic's values, d_embed (may be NULL)
 * [num_agents][512] the trunk inputs of the actor (256) then the critic (256).
 * Caller-owned device buffers.  The network keeps its activation buffers and
 * grows them (cudaMalloc, after synchronising its stream) when num_agents
 * exceeds every earlier call's.  Asynchronous on the network's stream.
 * Errors: SF_ERR_INVALID_ARG, SF_ERR_OOM, SF_ERR_CUDA. */
sf_status sf_lf_forward(sf_lf_handle m, const float* d_obs, const int32_t* d_n_road, const int32_t* d_n_veh,
                        int num_agents, float* d_mean, float* d_value, float* d_embed);

/* Wait for the network's stream; SF_ERR_TIMEOUT if a bounded tensor-core wait
 * gave up since the last sync. */
sf_status sf_lf_sync(sf_lf_handle m);

/* The paper's control loop (Alg. 1: observe, act, simulate) with this
 * network: the full observation of the current state, the actor's action
 * means (and the critic's values) from it, then one sf_step on those actions
 * (throttle and brake rectified, steer scaled, as for any action).  Buffers of
 * the observation, counts and values are allocated by the first call on h.
 * Asynchronous on h's stream; lf must not run elsewhere meanwhile.
 * Errors: SF_ERR_STATE, SF_ERR_INVALID_ARG, SF_ERR_OOM, SF_ERR_CUDA. */
sf_status sf_step_lf(sf_handle h, sf_lf_handle lf, float dt, int substeps);

/* Device pointers to what the last sf_step_lf (or its captured graph) used:
 * the full observation [A][SF_FULL_OBS_DIM], its counts [A], the actions [A][3]
 * and the critic values [A] (library-owned, valid until sf_destroy / the next
 * sf_load_roads). */
typedef struct {
    float* obs;
    int32_t* n_road;
    int32_t* n_veh;
    float* actions;
    float* value;
    int32_t num_agents;
} sf_lf_outputs;
sf_status sf_lf_step_outputs(sf_handle h, sf_lf_outputs* out);

/* Capture sf_step_lf (then sf_reset(d_reset_mask) if not NULL) into a CUDA
 * graph on h's stream (not the legacy default stream); replay with
 * sf_graph_launch.  Buffers are allocated before the capture.
 * Errors: SF_ERR_STATE, SF_ERR_INVALID_ARG, SF_ERR_OOM, SF_ERR_CUDA. */
sf_status sf_graph_capture_lf(sf_handle h, sf_lf_handle lf, const uint8_t* d_reset_mask, float dt, int substeps,
                              sf_graph_handle* out);

/* ------------------------------------------------------------------------
 * On-device PPO (SceneFactory App. L, Tab. app_ppo_hparams; the training
 * loop of Alg. 1) with the tensor-core MLPs: an actor (320 inputs, 3 outputs:
 * the mean of a diagonal Gaussian policy whose log standard deviation is a
 * free 3-vector) and a critic (320 inputs, 1 output), both sf_mlp handles.
 * A rollout of `horizon` control steps of the world handle (which must be
 * created with SF_FLAG_AUTO_RESET so that done agents respawn) records per
 * step and agent the 320-value observation, the sampled action (mean + sigma
 * times a standard normal from a counter-hashed Box-Muller draw), its
 * log-probability, the mean, the critic's value, the reward and the done
 * flag.  An update computes GAE advantages and returns
 * (delta_t = r_t + gamma (1 - d_t) V_{t+1} - V_t, A_t = delta_t +
 * gamma lambda (1 - d_t) A_{t+1}), normalises the advantages over the
 * rollout, and runs `epochs` x `minibatches` steps of: the clipped surrogate
 * -min(ratio A, clip(ratio, 1 - clip, 1 + clip) A) + vf_coef (V - R)^2 -
 * ent_coef H, its gradients through both MLPs, the mean Gaussian KL to the
 * rollout policy (learning rate halved when KL > 2 kl_target, doubled when
 * KL < kl_target / 2, within [1e-6, 1e-2]), gradient clipping to a global
 * norm of max_grad_norm, and Adam.  Minibatch rows are an affine bijection
 * of the rollout rows, drawn per epoch from the seed.  All of it runs on the
 * world handle's stream; the MLPs must not be used elsewhere meanwhile.
 * ---------------------------------------------------------------------- */
typedef struct sf_ppo* sf_ppo_handle;
typedef struct {
    int32_t horizon;         /* rollout steps per update (App. L: 128)     */
    int32_t minibatches;     /* minibatches per epoch (16)                  */
    int32_t epochs;          /* learning epochs (5)                         */
    float lr;                /* initial learning rate (2.09e-4)             */
    float kl_target;         /* adaptive learning-rate KL target (0.01)     */
    float gamma;             /* discount (0.99)                             */
    float lam;               /* GAE lambda (0.98)                           */
    float clip;              /* clip epsilon (0.15)                         */
    float ent_coef;          /* entropy coefficient (3e-5)                  */
    float vf_coef;           /* value loss coefficient (1.0)                */
    float max_grad_norm;     /* gradient norm limit (1.0)                   */
    float init_log_std;      /* initial log standard deviation (0)          */
    float dt;                /* control step (1/30 s)                       */
    int32_t substeps;        /* physics substeps per control step (4)       */
    uint64_t seed;           /* sampling and minibatch draws                */
} sf_ppo_config;

/* The paper's values above. */
void sf_ppo_default_config(sf_ppo_config* cfg);

/* Rollout buffers (library-owned device memory, valid until sf_ppo_destroy),
 * indexed [t][agent]: obs [T][A][320], actions and mean [T][A][3], logp,
 * reward, advantage, ret [T][A] float32, done [T][A] uint8, value [T + 1][A]
 * (the last row bootstraps GAE).  advantage / ret hold the last update's
 * normalised advantages and returns. */
typedef struct {
    float* obs;
    float* actions;
    float* mean;
    float* logp;
    float* value;
    float* reward;
    uint8_t* done;
    float* advantage;
    float* ret;
    int32_t horizon;
    int32_t num_agents;
    int32_t minibatch_rows;  /* floor(horizon * agents / minibatches) rounded down to a multiple of 8 */
} sf_ppo_rollout;

/* Allocates the rollout (horizon x agents rows) and the minibatch buffers.
 * Errors: SF_ERR_INVALID_ARG (MLP shapes, configuration), SF_ERR_STATE (no
 * roads), SF_ERR_OOM. */
sf_status sf_ppo_create(sf_handle h, sf_mlp_handle actor, sf_mlp_handle critic, const sf_ppo_config* cfg,
                        sf_ppo_handle* out);
sf_status sf_ppo_destroy(sf_ppo_handle p);
const char* sf_ppo_last_error(sf_ppo_handle p);

/* One rollout of `horizon` steps from the world's current state.  Asynchronous. */
sf_status sf_ppo_collect(sf_ppo_handle p);

/* GAE and the epochs of minibatch updates on the last rollout.  h_stats (may
 * be NULL; synchronous when given) [6] receives the rollout's mean reward per
 * agent-step and, averaged over the minibatches, the policy loss, the value
 * loss, the KL, then the current learning rate and the mean gradient norm
 * before clipping.  Errors: SF_ERR_STATE (no rollout), SF_ERR_CUDA. */
sf_status sf_ppo_update(sf_ppo_handle p, float* h_stats);

/* The policy's log standard deviations [3] (synchronous). */
sf_status sf_ppo_log_std(sf_ppo_handle p, float* h_log_std);
sf_status sf_ppo_rollout_ptrs(sf_ppo_handle p, sf_ppo_rollout* out);

/* The loss and its gradients for `rows` given rows (rows % 8 == 0, at most
 * minibatch_rows) with the current parameters, without updating anything:
 * d_obs [rows][320], d_small [rows][12] = (action 3, rollout mean 3, rollout
 * log-probability, normalised advantage, return, 3 unused); d_mean [rows][3]
 * and d_value [rows] receive the actor / critic outputs, d_dmean [rows][3] and
 * d_dvalue [rows] the loss gradients with respect to them (any of these four
 * may be NULL), h_out [6] the gradient with respect to the three log-stds,
 * then the policy loss, the value loss (mean squared error, without vf_coef)
 * and the mean KL to the last rollout's policy.  Synchronous. */
sf_status sf_ppo_loss_grads(sf_ppo_handle p, const float* d_obs, const float* d_small, int rows, float* d_mean,
                            float* d_value, float* d_dmean, float* d_dvalue, float* h_out);

/* PPO on the paper's own network (SceneFactory Alg. 1 with App. E and App. L):
 * the late-fusion actor-critic `lf` (sf_lf_create) on the full observation
 * (sf_observe_full), trained in place.  The engine takes lf's current
 * parameters (their last three, the log standard deviations, start the
 * policy's), keeps its own fp32 masters with Adam moments and, after every
 * update, writes the trained weights back into lf's device copies, so that
 * sf_lf_forward and the next rollout use them (sf_lf_get_params keeps
 * returning the parameters last set from the host; sf_ppo_lf_params returns
 * the trained ones).  Per rollout step the engine observes the full
 * observation and its group counts, runs lf, samples and steps; the rollout
 * buffers' obs are then [T][A][SF_FULL_OBS_DIM].  Every other part of the
 * update is the MLP engine's (GAE, the clipped loss, adaptive KL learning
 * rate, norm clipping, Adam).  The backward of each masked max-pool passes a
 * feature's gradient to the slot that held the maximum (the lowest slot on
 * ties) and recomputes that slot's first layer; the weight gradients are
 * sums in a fixed order, so two runs give bit-identical weights.  Each
 * minibatch step of sf_ppo_update waits once on its stream for the number of
 * distinct maximising slots (the row count of the set encoders' backward
 * products), so the update cannot be captured into a CUDA graph.
 * Errors: SF_ERR_INVALID_ARG (configuration), SF_ERR_STATE (no roads),
 * SF_ERR_OOM.  lf must not be used on another stream while the engine runs. */
sf_status sf_ppo_create_lf(sf_handle h, sf_lf_handle lf, const sf_ppo_config* cfg, sf_ppo_handle* out);

/* Gradient of L = sum(d_dmean * mean) + sum(d_dvalue * value) with respect to
 * every parameter of the engine's late-fusion network at its current
 * parameters, for `rows` observation rows (rows % 8 == 0): d_obs
 * [rows][SF_FULL_OBS_DIM], d_n_road / d_n_veh [rows] int32, d_dmean [rows][3],
 * d_dvalue [rows]; d_mean [rows][3] / d_value [rows] receive the training
 * forward's outputs (may be NULL when rows <= the minibatch rows); d_argmax
 * (may be NULL) [2 groups: road, vehicles][2 networks: actor, critic][rows][96]
 * uint16 receives the slot each pooled feature's gradient went to (the first
 * maximising slot as the forward computed it; 0xFFFF for an empty group).  h_grads
 * [n == sf_lf_num_params()] receives the gradient in sf_lf_set_params' layout
 * (the three log-std entries zero).  Updates nothing.  Synchronous.
 * Errors: SF_ERR_INVALID_ARG (an MLP-mode engine, NULL buffers, sizes). */
sf_status sf_ppo_lf_grads(sf_ppo_handle p, const float* d_obs, const int32_t* d_n_road, const int32_t* d_n_veh,
                          int rows, const float* d_dmean, const float* d_dvalue, float* d_mean, float* d_value,
                          uint16_t* d_argmax, float* h_grads, size_t n);

/* The late-fusion engine's trained parameters in sf_lf_set_params' layout,
 * log standard deviations included (h_params [n == sf_lf_num_params()]).
 * Synchronous. */
sf_status sf_ppo_lf_params(sf_ppo_handle p, float* h_params, size_t n);

/* Number of agents and worlds of the loaded roads (0 before sf_load_roads). */
int32_t sf_num_agents(sf_handle h);
int32_t sf_num_worlds(sf_handle h);

/* Message of the last failed call on h (or of the last sf_create failure when
 * h is NULL).  The string is owned by the library. */
const char* sf_last_error(sf_handle h);

/* Library version string. */
const char* sf_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SF_H */
