"""Learned half-resolution evolution (the learned corrector on top of the
plain method): driver code only - every arithmetic step is a call into
libbssn (RK4 steps, restriction, prolongation, constraints, the corrector's
tensor-core kernels); PyTorch only holds device buffers.

Pairs (a coarse step vs the restricted fine step) come from fine-grid
trajectories f_0, f_1, ... of the plain method with dt_f = dt_c / 2:
    input  = coarse_step(R(f_k))        (R = 2:1 restriction)
    target = R(f_{k+2})
and the network learns target - input. At run time a step is
    y_plain = coarse_step(y);  y_learned = y_plain + correction(y_plain)
and it falls back to the fine method (prolong y, two fine steps, restrict,
applied as an increment to y: fallback_step) when the Hamiltonian-constraint
L2 of y_learned exceeds `fallback_factor` times that of y_plain.
"""
import numpy as np
import torch

from . import binding as B
from . import inputs

NV = 24
CH = 32


class Problem:
    """One evolution setting shared by the coarse and the fine grid: a
    Brill-Lindquist pair on [-8, 8]^3 with static ghosts, or a gauge wave on
    [-0.5, 0.5]^3 with periodic ghosts."""

    def __init__(self, kind, nc, g=4, masses=(0.5, 0.5), separation=3.0, amplitude=0.05, order=4):
        self.kind = kind
        self.nc, self.nf, self.g = nc, 2 * nc, g
        self.params = B.make_params(fd_order=order, ko_eps=0.1, lapse=0, shift=0, eta=2.0)
        if kind == "bl":
            lo, hi = -8.0, 8.0
            centers = ((-separation / 2, 0.0, 0.0), (separation / 2, 0.0, 0.0))
            self.uc, hc = inputs.brill_lindquist(nc, g, lo=lo, hi=hi, masses=masses, centers=centers)
            self.uf, hf = inputs.brill_lindquist(2 * nc, g, lo=lo, hi=hi, masses=masses, centers=centers)
            self.bc = 1
        else:
            self.uc, hc = inputs.gauge_wave(nc, g, amplitude=amplitude, noise=0.0)
            self.uf, hf = inputs.gauge_wave(2 * nc, g, amplitude=amplitude, noise=0.0)
            self.bc = 0
        self.gc = B.make_grid(nc, ghost=g, dx=hc)
        self.gf = B.make_grid(2 * nc, ghost=g, dx=hf)
        self.dt_c = 0.25 * hc
        self.dt_f = 0.5 * self.dt_c


class Stepper:
    """Device buffers and plain steps for one Problem. The coarse steps use
    `prec`; the fine steps use `fine_prec` (default: the same)."""

    def __init__(self, prob, prec=B.FP64, fine_prec=None):
        self.p = prob
        self.prec = prec
        self.fine_prec = prec if fine_prec is None else fine_prec
        self.src_c = B.upload(prob.uc, prob.gc)
        self.src_f = B.upload(prob.uf, prob.gf)
        self.bufs_c = B.alloc_state(prob.gc, n=3)
        self.bufs_f = B.alloc_state(prob.gf, n=3)
        self.work_c = B.alloc_work(prob.gc, prob.params, prec)
        self.work_f = B.alloc_work(prob.gf, prob.params, self.fine_prec)
        self.work_con = B.alloc_work(prob.gc, prob.params, B.FP64)
        self.ko_buf = self.zero = None

    def coarse_step(self, state):
        B.rk4_step(self.p.gc, self.p.params, self.prec, self.p.dt_c, self.p.bc, self.src_c, state, self.bufs_c,
                   self.work_c)

    def fine_step(self, state):
        B.rk4_step(self.p.gf, self.p.params, self.fine_prec, self.p.dt_f, self.p.bc, self.src_f, state, self.bufs_f,
                   self.work_f)

    def step_change(self, after, before):
        """Per-variable RMS over interior points of a coarse step's change."""
        return B.rms_diff(self.p.gc, after, before, self.work_con)

    def roughness(self, after, before=None):
        """Per-variable RMS over interior points of the Kreiss-Oliger operator
        applied to a coarse state (its 2r-th undivided differences over h): a
        measure of the coarse grid's local truncation error, computed from
        the state alone."""
        if self.ko_buf is None:
            self.ko_buf = B.alloc_state(self.p.gc)
            self.zero = torch.zeros_like(self.ko_buf)
        B.ko_dissipation(self.p.gc, self.p.params, B.FP64, after, self.ko_buf)
        return B.rms_diff(self.p.gc, self.ko_buf, self.zero, self.work_con)

    def restrict(self, fine, coarse):
        B.restrict(self.p.gf, fine, self.p.gc, coarse)
        B.fill_ghosts(self.p.gc, self.p.bc, self.src_c if self.p.bc == 1 else None, coarse)

    def prolong(self, coarse, fine):
        B.fill_ghosts(self.p.gc, self.p.bc, self.src_c if self.p.bc == 1 else None, coarse)
        B.prolong(self.p.gc, coarse, self.p.gf, fine)
        B.fill_ghosts(self.p.gf, self.p.bc, self.src_f if self.p.bc == 1 else None, fine)

    def ham_l2(self, state):
        l2, mx, st = B.hamiltonian(self.p.gc, self.p.params, state, self.work_con)
        return l2 if st == B.OK else float("inf")


def trajectory_pairs(stepper, nsteps, measure=None):
    """Coarse pairs (input, target, size) along one fine trajectory of
    nsteps + 2 fine steps: input and target are device states; size is the
    per-variable vector (numpy, 24) that Stepper.<measure>(input, R(f_k))
    returns for the coarse step's output, or None without a measure."""
    p = stepper.p
    f = stepper.src_f.clone()
    restricted = []
    pairs = []
    for k in range(nsteps + 2):
        c = B.alloc_state(p.gc)
        stepper.restrict(f, c)
        restricted.append(c)
        if k >= 2:
            x = restricted[k - 2].clone()
            stepper.coarse_step(x)
            size = getattr(stepper, measure)(x, restricted[k - 2]) if measure else None
            pairs.append((x, restricted[k], size))
            restricted[k - 2] = None
        stepper.fine_step(f)
    return pairs


def step_reference(pairs):
    """Per-variable reference of the pairs' size vectors: their RMS over the
    pairs (floored so that it is never zero)."""
    S = np.array([q[2] for q in pairs])
    ref = np.sqrt((S ** 2).mean(axis=0))
    return np.maximum(ref, 1e-12 + 1e-6 * ref.max())


def step_scale(change, ref, floor=1e-4):
    """Output scale of one sample: its size vector relative to the
    reference, per variable, floored at `floor`."""
    return np.maximum(np.asarray(change) / ref, floor)


def default_scales(pairs, grid):
    """Per-variable input offset/scale and output scale from a few pairs
    (host statistics of the interior): offset = mean, scale = 1/std
    (floored), output scale = 1/rms(target - input)."""
    xs, ds = [], []
    for x, t, *_ in pairs:
        a = B.download(x, grid)[:, grid.ghost:-grid.ghost, grid.ghost:-grid.ghost, grid.ghost:-grid.ghost]
        b = B.download(t, grid)[:, grid.ghost:-grid.ghost, grid.ghost:-grid.ghost, grid.ghost:-grid.ghost]
        xs.append(a.reshape(NV, -1))
        ds.append((b - a).reshape(NV, -1))
    X = np.concatenate(xs, axis=1)
    D = np.concatenate(ds, axis=1)
    off = X.mean(axis=1)
    sd = X.std(axis=1)
    in_scale = 1.0 / np.maximum(sd, 1e-3 * np.maximum(np.abs(off), 1.0))
    rms = np.sqrt((D ** 2).mean(axis=1))
    out_scale = 1.0 / np.maximum(rms, 1e-12 + 1e-3 * rms.max())
    return off, in_scale, out_scale


class Dataset:
    """Packed BF16 pairs on the device. With step_ref, each pair's target is
    taken relative to its own coarse step's change (step_scale)."""

    def __init__(self, corrector, n, step_ref=None):
        self.c = corrector
        self.n = n
        self.step_ref = step_ref
        self.x, self.t = [], []

    def add(self, pairs, grid):
        for inp, tgt, *rest in pairs:
            xb = torch.empty((self.n ** 3, CH), dtype=torch.bfloat16, device="cuda")
            tb = torch.empty_like(xb)
            if self.step_ref is not None:
                B.corrector_set_step_scale(self.c, step_scale(rest[0], self.step_ref))
            B.corrector_pack(self.c, grid, inp, tgt, xb, tb)
            self.x.append(xb)
            self.t.append(tb)

    def __len__(self):
        return len(self.x)


def train(corrector, data, epochs, batch, lr, seed=0, lr_final=None, log=None):
    """Adam over shuffled mini-batches; lr decays geometrically to lr_final.
    Returns the list of per-step losses."""
    rng = np.random.default_rng(seed)
    n = len(data)
    steps = epochs * (n // batch)
    lr_final = lr if lr_final is None else lr_final
    losses = []
    k = 0
    for ep in range(epochs):
        order = rng.permutation(n)
        for b0 in range(0, n - batch + 1, batch):
            idx = order[b0:b0 + batch]
            rate = lr * (lr_final / lr) ** (k / max(1, steps - 1))
            losses.append(B.corrector_train_step_raw(corrector, [data.x[i] for i in idx], [data.t[i] for i in idx],
                                                     rate))
            k += 1
        if log:
            log(f"epoch {ep}: mean loss {np.mean(losses[-(n // batch):]):.4e}")
    return losses


def fallback_step(stepper, before, out):
    """The plain fine method over one coarse step, as an increment: out =
    y + R(F F P y) - R(P y) for y = before (P prolongation, F a fine step,
    R restriction). Restricting the prolonged state does not give y back
    exactly (a fourth-order difference of the state itself, large against
    one step's change), so only the fine method's change is taken from the
    fine grid."""
    p = stepper.p
    fine = B.alloc_state(p.gf)
    stepper.prolong(before, fine)
    base = B.alloc_state(p.gc)
    stepper.restrict(fine, base)
    stepper.fine_step(fine)
    stepper.fine_step(fine)
    stepper.restrict(fine, out)
    B.add_difference(p.gc, before, out, base, out)
    B.fill_ghosts(p.gc, p.bc, stepper.src_c if p.bc == 1 else None, out)


def learned_step(stepper, corrector, state, fallback_factor=2.0, scratch=None, step_ref=None, measure="roughness"):
    """One learned coarse step in place. Returns (used_fallback, H_learned,
    H_plain). With step_ref, the correction is scaled by this step's own
    size vector (Stepper.<measure>, as the training targets were)."""
    p = stepper.p
    before = state.clone() if scratch is None else scratch.copy_(state)
    stepper.coarse_step(state)
    h_plain = stepper.ham_l2(state)
    if step_ref is not None:
        B.corrector_set_step_scale(corrector, step_scale(getattr(stepper, measure)(state, before), step_ref))
    B.corrector_apply(corrector, p.gc, state)
    B.fill_ghosts(p.gc, p.bc, stepper.src_c if p.bc == 1 else None, state)
    h_learned = stepper.ham_l2(state)
    if not (h_learned <= fallback_factor * h_plain):
        fallback_step(stepper, before, state)
        return True, h_learned, h_plain
    return False, h_learned, h_plain


def evaluate(stepper, corrector, nsteps, fallback_factor=2.0, step_ref=None, measure="roughness"):
    """Evolve nsteps coarse steps three ways - plain coarse, learned, and the
    fine method restricted - and return the errors of plain and learned
    against the restricted fine solution (RMS over interior points and
    variables, each variable normalised by its RMS change over the run), the
    Hamiltonian-constraint L2 of each, and the fallback count."""
    p = stepper.p
    g = p.g
    fine = stepper.src_f.clone()
    plain = B.alloc_state(p.gc)
    stepper.restrict(fine, plain)
    learned = plain.clone()
    start = plain.clone()
    ref = B.alloc_state(p.gc)
    fallbacks = 0
    for _ in range(nsteps):
        stepper.coarse_step(plain)
        fb, _, _ = learned_step(stepper, corrector, learned, fallback_factor, step_ref=step_ref, measure=measure)
        fallbacks += int(fb)
        stepper.fine_step(fine)
        stepper.fine_step(fine)
    stepper.restrict(fine, ref)
    I = (slice(None),) + (slice(g, -g),) * 3
    r = B.download(ref, p.gc)[I].reshape(NV, -1)
    s0 = B.download(start, p.gc)[I].reshape(NV, -1)
    change = np.sqrt(((r - s0) ** 2).mean(axis=1))
    norm = np.maximum(change, 1e-12 + 1e-6 * change.max())

    def err(x):
        a = B.download(x, p.gc)[I].reshape(NV, -1)
        return float(np.sqrt((((a - r) / norm[:, None]) ** 2).mean()))

    return dict(err_plain=err(plain), err_learned=err(learned), ham_plain=stepper.ham_l2(plain),
                ham_learned=stepper.ham_l2(learned), ham_fine=stepper.ham_l2(ref), fallbacks=fallbacks)
