"""Plain CPU oracle of the lbest-ring particle swarm optimiser (Sec. III) and of its random numbers.

TEST INFRASTRUCTURE ONLY (see the package docstring).

PSO as used by the paper (Sec. III): particles move in a search box under a social and a
cognitive attraction, lbest topology on a ring of particle indices, a fixed number of iterations,
best-of-M independent runs with independent random streams. The paper defers the remaining
details to earlier work; the readings taken here (the standard settings of that earlier lbest
PSO work, stated in full so that the device code can be checked against them):

  * positions normalised to [0, 1]^4; alpha = 2 pi x0, delta = pi (x1 - 1/2),
    tau0 = lo + (hi - lo) x2, tau1.5 = lo + (hi - lo) x3;
  * inertia w decreasing linearly from w_start to w_end over the iterations, c1 = c2 = 2,
    every velocity component clamped to [-vmax, vmax];
  * ring neighbourhood = the particle and n_neighbours particles on each side; lbest = the best
    personal best in it (lowest index on ties);
  * "let them fly": a particle outside the box is not evaluated, its fitness is -inf;
  * initial x ~ U[0,1]^4, v = u' - x with u' ~ U[0,1]^4, then clamped;
  * one iteration = evaluate, update personal bests, update local bests, move.

Random numbers: Philox4x32-10 (Salmon et al., "Parallel random numbers: as easy as 1, 2, 3", SC'11),
counter (run, iteration, particle, stream) under key (seed lo, seed hi); uniforms (u + 1/2) 2^-32.
The velocity update is evaluated in binary64 in one fixed order without fused multiply-adds,
so that an implementation following the same order reproduces it bit for bit.
"""

import math

import numpy as np

M0, M1 = 0xD2511F53, 0xCD9E8D57
W0, W1 = 0x9E3779B9, 0xBB67AE85
MASK = 0xFFFFFFFF
INIT_ITER = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds on arrays: ctr (..., 4) uint32, key (..., 2) uint32 -> (..., 4) uint32."""
    c = np.asarray(ctr, dtype=np.uint64) & MASK
    k = np.asarray(key, dtype=np.uint64) & MASK
    c0, c1, c2, c3 = c[..., 0].copy(), c[..., 1].copy(), c[..., 2].copy(), c[..., 3].copy()
    k0, k1 = k[..., 0].copy(), k[..., 1].copy()
    for rnd in range(10):
        p0 = np.uint64(M0) * c0            # < 2^64, exact in uint64
        p1 = np.uint64(M1) * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & np.uint64(MASK)
        hi1, lo1 = p1 >> np.uint64(32), p1 & np.uint64(MASK)
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        if rnd < 9:
            k0 = (k0 + np.uint64(W0)) & np.uint64(MASK)
            k1 = (k1 + np.uint64(W1)) & np.uint64(MASK)
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def uniforms(run, it, particles, stream, seed):
    """(len(particles), 4) uniforms in (0, 1) for counter (run, it, p, stream)."""
    p = np.asarray(particles, dtype=np.uint64)
    ctr = np.stack([np.full_like(p, run), np.full_like(p, it), p, np.full_like(p, stream)], axis=-1)
    key = np.broadcast_to(np.array([seed & MASK, (seed >> 32) & MASK], dtype=np.uint64), ctr.shape[:-1] + (2,))
    u = philox4x32_10(ctr, key).astype(np.float64)
    return (u + 0.5) * 2.0 ** -32


class PsoConfig:
    def __init__(self, n_runs=8, n_particles=40, n_iter=2000, n_neighbours=1, seed=0,
                 box=(0.0, 2 * math.pi, -0.5 * math.pi, 0.5 * math.pi, 1.0, 2.0, 0.1, 0.2),
                 w_start=0.9, w_end=0.4, c1=2.0, c2=2.0, vmax=0.5):
        self.n_runs, self.n_particles, self.n_iter, self.n_neighbours = n_runs, n_particles, n_iter, n_neighbours
        self.seed = seed
        self.box = tuple(float(b) for b in box)
        self.w_start, self.w_end, self.c1, self.c2, self.vmax = w_start, w_end, c1, c2, vmax


def to_theta(cfg, x):
    """Normalised positions (..., 4) -> (alpha, delta, tau0, tau1.5)."""
    a0, a1, d0, d1, t0, t1, s0, s1 = cfg.box
    return np.stack([a0 + (a1 - a0) * x[..., 0], d0 + (d1 - d0) * x[..., 1],
                     t0 + (t1 - t0) * x[..., 2], s0 + (s1 - s0) * x[..., 3]], axis=-1)


def in_box(x):
    return np.all((x >= 0.0) & (x <= 1.0), axis=-1)


def inertia(cfg, it):
    if cfg.n_iter <= 1:
        return cfg.w_start
    return cfg.w_start + (cfg.w_end - cfg.w_start) * (float(it) / float(cfg.n_iter - 1))


class PsoState:
    """State of all runs: arrays of shape (n_runs, n_particles, ...)."""

    def __init__(self, cfg):
        r, p = cfg.n_runs, cfg.n_particles
        self.x = np.zeros((r, p, 4))
        self.v = np.zeros((r, p, 4))
        self.pbest_x = np.zeros((r, p, 4))
        self.pbest_f = np.full((r, p), -np.inf)
        self.pbest_tc = np.full((r, p), -1, dtype=np.int64)


def init_state(cfg):
    s = PsoState(cfg)
    idx = np.arange(cfg.n_particles)
    for run in range(cfg.n_runs):
        x = uniforms(run, INIT_ITER, idx, 0, cfg.seed)
        u = uniforms(run, INIT_ITER, idx, 1, cfg.seed)
        s.x[run] = x
        s.v[run] = np.minimum(np.maximum(u - x, -cfg.vmax), cfg.vmax)
        s.pbest_x[run] = x
    return s


def local_best(cfg, pbest_f):
    """Index of the best personal best in each particle's ring neighbourhood (lowest index on ties)."""
    p = pbest_f.shape[-1]
    out = np.empty(pbest_f.shape, dtype=np.int64)
    for run in range(pbest_f.shape[0]):
        for i in range(p):
            best = None
            for q in sorted({(i + d) % p for d in range(-cfg.n_neighbours, cfg.n_neighbours + 1)}):
                if best is None or pbest_f[run, q] > pbest_f[run, best]:
                    best = q
            out[run, i] = best
    return out


def update(cfg, s, it, fitness, tc):
    """One PSO iteration after the fitness of the current positions is known (fitness -inf for
    particles outside the box): personal bests, local bests, then the move."""
    inside = in_box(s.x)
    f = np.where(inside, fitness, -np.inf)
    better = f > s.pbest_f
    s.pbest_f = np.where(better, f, s.pbest_f)
    s.pbest_x = np.where(better[..., None], s.x, s.pbest_x)
    s.pbest_tc = np.where(better, tc, s.pbest_tc)
    lb = local_best(cfg, s.pbest_f)
    lbest_x = np.take_along_axis(s.pbest_x, lb[..., None].repeat(4, axis=-1), axis=1)
    w = inertia(cfg, it)
    idx = np.arange(cfg.n_particles)
    for run in range(cfg.n_runs):
        r1 = uniforms(run, it, idx, 0, cfg.seed)
        r2 = uniforms(run, it, idx, 1, cfg.seed)
        x, v = s.x[run], s.v[run]
        # v' = ((w v + (c1 r1) (pbest - x)) + (c2 r2) (lbest - x)), element-wise binary64, this order
        a = w * v
        b = (cfg.c1 * r1) * (s.pbest_x[run] - x)
        c = (cfg.c2 * r2) * (lbest_x[run] - x)
        vn = (a + b) + c
        vn = np.minimum(np.maximum(vn, -cfg.vmax), cfg.vmax)
        s.v[run] = vn
        s.x[run] = x + vn
    return s


def run_search(cfg, fitness_fn):
    """Full search with a fitness function theta (n, 4) -> (fitness (n,), tc (n,)).
    Returns per run (best fitness, best theta, best tc) and the final state."""
    s = init_state(cfg)
    for it in range(cfg.n_iter):
        flat = s.x.reshape(-1, 4)
        inside = in_box(flat)
        fit = np.full(flat.shape[0], -np.inf)
        tcs = np.full(flat.shape[0], -1, dtype=np.int64)
        if np.any(inside):
            f, t = fitness_fn(to_theta(cfg, flat[inside]))
            fit[inside] = f
            tcs[inside] = t
        update(cfg, s, it, fit.reshape(cfg.n_runs, cfg.n_particles), tcs.reshape(cfg.n_runs, cfg.n_particles))
    best = np.argmax(s.pbest_f, axis=1)
    res = [(s.pbest_f[r, best[r]], to_theta(cfg, s.pbest_x[r, best[r]]), s.pbest_tc[r, best[r]])
           for r in range(cfg.n_runs)]
    return res, s
