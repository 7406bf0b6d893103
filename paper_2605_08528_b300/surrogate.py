"""Training and evaluation driver of the learned dynamics surrogate.

Everything numeric runs in the library's kernels (collection of transitions
from the physics step, statistics, Adam through the tensor-core MLP, the
surrogate step); this module only sequences the C-ABI calls and holds the
device buffers.
"""
from __future__ import annotations

import numpy as np

from . import sf, synth


def collect_and_train(scene, transitions=10_000_000, train_steps=60000, batch=8192, lr=3e-3, seed=1, stream=None,
                      max_steps=100_000):
    """Collect up to `transitions` physics transitions of gated agents on `scene`
    (smooth random actions, automatic resets) and train a new surrogate.
    Returns (surrogate handle, rows used, final loss)."""
    import torch
    W = sf.World(scene, seed=seed, flags=sf.FLAG_AUTO_RESET, stream=stream)
    dev = torch.device("cuda")
    s = sf.sf_surrogate_create(stream)
    with torch.cuda.stream(stream) if stream is not None else _null():
        sf.sf_reset(W.h, torch.ones(W.A, dtype=torch.uint8, device=dev))
        ring = 256
        acts = torch.as_tensor(synth.ou_actions(W.A, ring, seed=seed + 100), device=dev)
        dx = torch.empty((transitions, sf.SURR_IN), dtype=torch.float32, device=dev)
        dy = torch.empty((transitions, sf.SURR_OUT), dtype=torch.float32, device=dev)
        cnt = torch.zeros(1, dtype=torch.int64, device=dev)
        t = 0
        while t < max_steps:
            sf.sf_surrogate_collect(W.h, s, acts[t % ring], dx, dy, transitions, cnt)
            t += 1
            if t % 64 == 0 and int(cnt.item()) >= transitions:
                break
        n = min(int(cnt.item()), transitions)
    W.close()
    loss = sf.sf_surrogate_train(s, dx, dy, n, batch=batch, steps=train_steps, lr=lr, seed=seed)
    del dx, dy
    return s, n, loss


def rollout_error(s, scene, steps=30, warm=10, seed=5, stream=None, segments=1):
    """Position error after `steps` control steps between the surrogate path and
    the FP32 physics path started from identical states with identical actions
    (lone agents).  The physics world runs on through `segments` back-to-back
    windows; each window starts the surrogate world from a copy of the physics
    world's state, so every agent gives `segments` start states.  Returns
    (errors [segments * A], fraction of agent-steps on the surrogate)."""
    import torch
    dev = torch.device("cuda")
    W1 = sf.World(scene, seed=seed, flags=sf.FLAG_INVINCIBLE, stream=stream)
    W2 = sf.World(scene, seed=seed, flags=sf.FLAG_INVINCIBLE, stream=stream)
    acts = torch.as_tensor(synth.ou_actions(W1.A, warm + segments * steps, seed=seed + 1), device=dev)
    sf.sf_reset(W1.h, torch.ones(W1.A, dtype=torch.uint8, device=dev))
    for t in range(warm):
        sf.sf_step(W1.h, acts[t])
    used = 0
    errs = []
    for k in range(segments):
        F, I, _ = sf.sf_get_state(W1.h)
        sf.sf_set_state(W2.h, F, I)
        for t in range(steps):
            a = acts[warm + k * steps + t]
            sf.sf_step(W1.h, a)
            sf.sf_step_surrogate(W2.h, s, a)
            used += sf.sf_surrogate_audit(W2.h)[1]
        F1, _, _ = sf.sf_get_state(W1.h)
        F2, _, _ = sf.sf_get_state(W2.h)
        errs.append(np.linalg.norm(F1[:, :3] - F2[:, :3], axis=1))
    W1.close()
    W2.close()
    return np.concatenate(errs), used / float(segments * steps * W1.A)


class _null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False
