"""The DOT training loop (Algorithm 1) on top of the C ABI.

One optimisation step on a batch of stochastic ray samples (Sec. 4.1):
    forward render with the training signal fused (Sec. 3.1: Q accumulates over the epoch),
    MSE loss and dL/dC, backward into FP32 gradients that also flags the leaves it touches -- by
    default all three in one launch (dot_render_forward_backward_mse), else as dot_render_forward,
    dot_mse_grad and dot_render_backward -- then the RMSProp update fused with
    zeroing the gradients (Sec. 3.3, learning rates of Sec. 4.1): by default only over the touched
    leaves, with the pure decay of the others deferred (dot_rmsprop_step_sparse, the same update
    up to FP32 rounding), else over every leaf (dot_rmsprop_step).
Every T epochs (Algorithm 1) the tree is refined from the accumulated signal: pruning with
threshold tau (optionally recursive, merging parents upward while groups still qualify, the
merged signal being the sum -- or max -- of the children's), then sampling of the top-gamma
fraction (Sec. 3.2), with the RMSProp state carried through the refine (mean of merged children,
copies for sampled children).

Every step runs in libdot's kernels; this module only holds the device buffers and sequences the
calls.
"""
from __future__ import annotations

import time
from typing import Callable, Iterable, List, Optional, Tuple

import torch

from . import dot


class Trainer:
    def __init__(self, tree: dot.Octree, opts: dot.dot_render_opts,
                 rms: Optional[dot.dot_rmsprop_opts] = None,
                 signal_mode: int = dot.DOT_SIGNAL_SUM_ALPHA, stream=None, sparse: bool = True,
                 fused: bool = True):
        self.tree = tree
        self.sparse = sparse
        self.fused = fused
        self.step_no = 0
        self.opts = dot.render_opts(background=tuple(opts.background), eps_T=opts.eps_T,
                                    color_act=opts.color_act, signal_mode=signal_mode,
                                    precision=opts.precision, max_steps=opts.max_steps)
        self.rms = rms if rms is not None else dot.rmsprop_opts()
        self.signal_mode = signal_mode
        self.stream = stream
        self.loss_sum = torch.zeros(1, dtype=torch.float64, device="cuda")
        self._batch = 0
        self._alloc_leaf_state(zero_ms=True)

    # ---- per-leaf state --------------------------------------------------------------------
    def _alloc_leaf_state(self, zero_ms: bool):
        inf = self.tree.info()
        L, K = int(inf.n_leaves), int(inf.n_coeffs)
        self.L, self.K = L, K
        self.grad_sigma = torch.zeros(L, dtype=torch.float32, device="cuda")
        self.grad_sh = torch.zeros(L, 3, K, dtype=torch.float32, device="cuda")
        self.signal = torch.zeros(L, dtype=torch.float32, device="cuda")
        if zero_ms:
            self.ms_sigma = torch.zeros(L, dtype=torch.float32, device="cuda")
            self.ms_sh = torch.zeros(L, 3, K, dtype=torch.float32, device="cuda")
        self._alloc_sparse_state()

    def _alloc_sparse_state(self):
        L = self.L
        self.touched = torch.zeros(L, dtype=torch.uint8, device="cuda")
        self.last_step = torch.full((L,), self.step_no, dtype=torch.int32, device="cuda")
        self.work = torch.empty(L + 1, dtype=torch.int32, device="cuda")

    def _buffers(self, R: int):
        if self._batch != R:
            self.rgb = torch.empty(R, 3, dtype=torch.float32, device="cuda")
            self.grad_rgb = torch.empty(R, 3, dtype=torch.float32, device="cuda")
            self._batch = R

    # ---- Algorithm 1, optimization ---------------------------------------------------------
    def step(self, rays: dot.dot_rays, target: torch.Tensor):
        """One optimisation step on `rays` against `target` [R, 3]; the batch MSE is added to
        self.loss_sum (device float64)."""
        R = dot.n_rays_of(rays)
        self._buffers(R)
        s = self.stream
        sig = self.signal if self.signal_mode != dot.DOT_SIGNAL_NONE else None
        touched = self.touched if self.sparse else None
        if self.fused:
            dot.dot_render_forward_backward_mse(self.tree, rays, self.opts, target, self.rgb,
                                                self.grad_rgb, self.grad_sigma, self.grad_sh,
                                                self.loss_sum, sig, touched, stream=s)
        else:
            dot.dot_render_forward(self.tree, rays, self.opts, self.rgb, None, sig, stream=s)
            dot.dot_mse_grad(self.rgb, target, self.grad_rgb, self.loss_sum, stream=s)
            plain = dot.render_opts(background=tuple(self.opts.background), eps_T=self.opts.eps_T,
                                    color_act=self.opts.color_act, precision=self.opts.precision,
                                    max_steps=self.opts.max_steps)
            dot.dot_render_backward(self.tree, rays, plain, self.grad_rgb, self.rgb,
                                    self.grad_sigma, self.grad_sh, touched=touched, stream=s)
        self.step_no += 1
        if self.sparse:
            dot.dot_rmsprop_step_sparse(self.tree, self.grad_sigma, self.grad_sh, self.ms_sigma,
                                        self.ms_sh, self.touched, self.last_step, self.step_no,
                                        self.work, self.rms, stream=s)
        else:
            dot.dot_rmsprop_step(self.tree, self.grad_sigma, self.grad_sh, self.ms_sigma,
                                 self.ms_sh, self.rms, stream=s)

    def flush(self):
        """Brings every leaf's RMSProp mean squares up to the current step (sparse mode)."""
        if self.sparse:
            dot.dot_rmsprop_flush(self.tree, self.ms_sigma, self.ms_sh, self.last_step,
                                  self.step_no, self.rms, stream=self.stream)

    # ---- Algorithm 1, pruning and sampling -------------------------------------------------
    def refine(self, tau: float, gamma: float, depth_cap: int, recursive: bool = False,
               prune_mode: int = dot.DOT_SELECT_THRESHOLD,
               sample_mode: int = dot.DOT_SELECT_FRACTION, canonical: bool = False) -> dict:
        """Prunes leaves with signal <= tau (recursively when asked), then samples the top-gamma
        fraction by the signal (Algorithm 1); with `canonical` the tree is then renumbered in
        breadth-first Morton order (the RMSProp state follows).  Returns the plan of each pass."""
        merge = dot.DOT_MERGE_MAX if self.signal_mode == dot.DOT_SIGNAL_MAX_WEIGHT else dot.DOT_MERGE_SUM
        self.flush()
        passes = []
        while True:
            pm, sm = self._marks(dot.select_opts(prune_mode, tau, dot.DOT_SELECT_NONE, 0.0))
            plan = dot.dot_refine_plan(self.tree, pm, sm, depth_cap, stream=self.stream)
            if plan["n_pruned_groups"] == 0:
                break
            self._apply(pm, sm, depth_cap, plan, merge)
            passes.append(plan)
            if not recursive:
                break
        pm, sm = self._marks(dot.select_opts(dot.DOT_SELECT_NONE, 0.0, sample_mode, gamma))
        plan = dot.dot_refine_plan(self.tree, pm, sm, depth_cap, stream=self.stream)
        if plan["n_sampled"] > 0:
            self._apply(pm, sm, depth_cap, plan, merge)
            passes.append(plan)
        if canonical:
            perm = torch.empty(self.L, dtype=torch.int32, device="cuda")
            ms_sigma, ms_sh = torch.empty_like(self.ms_sigma), torch.empty_like(self.ms_sh)
            dot.dot_tree_canonicalize(self.tree, perm, [(self.ms_sigma, ms_sigma),
                                                        (self.ms_sh, ms_sh)], stream=self.stream)
            self.ms_sigma, self.ms_sh = ms_sigma, ms_sh
            self.leaf_perm = perm
        # a new stabilisation interval starts: fresh signal and gradients
        self.grad_sigma = torch.zeros(self.L, dtype=torch.float32, device="cuda")
        self.grad_sh = torch.zeros(self.L, 3, self.K, dtype=torch.float32, device="cuda")
        self.signal = torch.zeros(self.L, dtype=torch.float32, device="cuda")
        self._alloc_sparse_state()
        return {"passes": passes, "n_leaves": self.L, "n_nodes": self.tree.n_nodes}

    # ---- Algorithm 1, the whole loop ----------------------------------------------------------
    def fit(self, epoch_batches: Callable[[int], Iterable[Tuple[dot.dot_rays, torch.Tensor]]],
            epochs: int, T: int, tau: float, gamma: float, depth_cap: int,
            recursive: bool = True, prune_mode: int = dot.DOT_SELECT_THRESHOLD,
            sample_mode: int = dot.DOT_SELECT_FRACTION, canonical: bool = False,
            on_refine: Optional[Callable[[int, dict], None]] = None) -> List[float]:
        """Algorithm 1: for epoch i = 1..epochs, one optimisation pass over
        `epoch_batches(i)` -- the caller's (rays, target) batches in that epoch's permuted order --
        accumulating the signal Q, then, when i is a multiple of T, pruning with tau (recursively
        when asked) and sampling the top-gamma fraction.  `on_refine(i, plan)` is called after each
        refine (the leaf numbering has changed: a caller holding per-leaf arrays remaps them with
        self.leaf_map).  Returns the mean batch MSE of every epoch; the wall time of every refine
        (device work included) is appended to self.refine_ms."""
        losses = []
        self.refine_ms = []
        for i in range(1, epochs + 1):
            self.loss_sum.zero_()
            n = 0
            for rays, target in epoch_batches(i):
                self.step(rays, target)
                n += 1
            losses.append(float(self.loss_sum.item()) / max(n, 1))
            if i % T == 0:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                plan = self.refine(tau, gamma, depth_cap, recursive=recursive,
                                   prune_mode=prune_mode, sample_mode=sample_mode,
                                   canonical=canonical)
                torch.cuda.synchronize()
                self.refine_ms.append((time.perf_counter() - t0) * 1e3)
                if on_refine is not None:
                    on_refine(i, plan)
        return losses

    def _marks(self, sel: dot.dot_select_opts):
        pm = torch.empty(self.L, dtype=torch.uint8, device="cuda")
        sm = torch.empty(self.L, dtype=torch.uint8, device="cuda")
        dot.dot_select_masks(self.tree, self.signal, sel, pm, sm, stream=self.stream)
        return pm, sm

    def _apply(self, pm, sm, depth_cap, plan, merge):
        Ln, K = plan["n_leaves"], self.K
        lm = torch.empty(Ln, dtype=torch.int32, device="cuda")
        ms_sigma = torch.empty(Ln, dtype=torch.float32, device="cuda")
        ms_sh = torch.empty(Ln, 3, K, dtype=torch.float32, device="cuda")
        signal = torch.empty(Ln, dtype=torch.float32, device="cuda")
        aux = [(self.ms_sigma, ms_sigma, dot.DOT_MERGE_MEAN), (self.ms_sh, ms_sh, dot.DOT_MERGE_MEAN),
               (self.signal, signal, merge)]
        dot.dot_refine_prune(self.tree, pm, sm, depth_cap, lm, aux, stream=self.stream)
        self.ms_sigma, self.ms_sh, self.signal = ms_sigma, ms_sh, signal
        self.leaf_map = lm
        self.L = Ln
