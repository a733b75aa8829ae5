"""Element-by-element comparison of the CUDA path with the FP64 oracle.

Floating point decides an integer in the Map: row i is violated when its
residual r_i = <a_i, x> - b_i is positive (Eq. 7 gives it a non-zero
slice; Eq. 8 counts it in h).  A row whose oracle residual lies within a
rigorous bound of the accumulation type's rounding error is "ambiguous":
either classification is correct.  The checks here

  * accept any h between the number of surely violated rows and that
    number plus the ambiguous rows;
  * compare every element y_j of the Reduce with the oracle's sum over the
    rows whose classification is fixed, within
        tol_rel * |y_ref_j| + B_j,
    B_j = sum_i [bound_i / n2_i + gamma_D (|r_i| + bound_i) / n2_i] |a_ij|
          + sum over ambiguous i of |r_i| / n2_i |a_ij|,
    i.e. the column's share of the residual errors, of the rounding of the
    slice sums over D levels, and of the ambiguous rows' slices;
  * compare every element of a step dx = x_{k+1} - x_k with the oracle's
    step from the same x_k (relaxed: lambda y / h with the kernel's h;
    ModAP: lambda y / ||y||), with the same per-element bound scaled by the
    step factor, and ||dx_gpu - dx_ref|| <= tol_rel ||dx_ref|| + ||bound||.

The tolerance tol_rel = 1e-5 is the stated per-iteration tolerance for
binary32 accumulation (1e-12 for binary64 storage).
"""
from __future__ import annotations

import math

import numpy as np

import oracle

# unit roundoff of the accumulation type per storage type
U = {"f64": 2.0 ** -53, "f32": 2.0 ** -24, "bf16": 2.0 ** -24, "fp8": 2.0 ** -24}
TOL = {"f64": 1e-12, "f32": 1e-5, "bf16": 1e-5, "fp8": 1e-5}


def gamma(k: int, u: float) -> float:
    """gamma_k = k u / (1 - k u): the relative bound of a k-level sum."""
    ku = k * u
    return ku / (1.0 - ku) if ku < 0.5 else float("inf")


def _abs_matvec(Aabs, v):
    """|A| v for non-negative v, in A's own type (binary32 sums of positive
    terms are within n u of the exact value: a margin of 1.01 covers it)."""
    if Aabs.dtype == np.float64:
        return Aabs @ v
    return (Aabs @ v.astype(Aabs.dtype)).astype(np.float64) * 1.01


def residual_bound(A, x, b, u, levels=64, Aabs=None):
    """|computed r_i - exact r_i| <= bound_i for a dot product summed over at
    most `levels` levels (per-thread sequential partial sums, warp tree, block
    sum): gamma_levels (sum_j |a_ij x_j| + |b_i|), with a factor 2 of slack.
    The row record's rounding of b0 and Av to the accumulation type and the
    fused tick term are a few units of |b_i|, covered by the same term."""
    if Aabs is None:
        Aabs = np.abs(np.asarray(A))
    return 2.0 * gamma(levels, u) * (_abs_matvec(Aabs, np.abs(np.asarray(x, np.float64)))
                                     + np.abs(b) + 1e-300)


def dot_levels(n: int, threads: int = 512) -> int:
    """Levels of a row's dot product in the dense Map kernels: each of at
    most `threads` threads sums its share of the row in order, then a warp
    tree and a block sum (with margin)."""
    return math.ceil(n / threads) + 32


def dense_y_depth(m: int, num_ctas: int) -> int:
    """Levels of the slice sums of the dense Map and Reduce: each CTA adds
    its ceil(m / G) rows in order, the reduce adds G partial rows in eight
    groups and the eight group sums, plus the rounding of the slice
    coefficient (1/||a_i||^2 and r_i / ||a_i||^2)."""
    g = max(1, min(m, num_ctas))
    return math.ceil(m / g) + math.ceil(g / 8) + 8 + 4


def num_sms() -> int:
    """SM count of the current CUDA device (the dense Map's grid size)."""
    import torch
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def to_accumulation(x, storage):
    """The iterate as the Map reads it: rounded to the accumulation type."""
    x = np.asarray(x, np.float64)
    return x if storage == "f64" else x.astype(np.float32).astype(np.float64)


class _Ref:
    """Classification of the rows and the per-column bound B; subclasses
    fill r, bound, n2, mr, y (oracle sum over the fixed rows) and B."""

    def _classify(self):
        r = self.mr["r"]
        self.amb = np.abs(r) <= self.bound
        self.sure = (r > 0) & ~self.amb
        self.h_sure = int(self.sure.sum())
        self.n_amb = int(self.amb.sum())

    def _weights(self):
        """(w1, w2): B_j = sum_i |a_ij| (w1_i + gamma_D(j) w2_i)."""
        r = self.mr["r"]
        cand = self.sure | self.amb
        w1 = np.zeros(r.shape[0])
        w2 = np.zeros(r.shape[0])
        w1[cand] = self.bound[cand] / self.n2[cand]
        w2[cand] = (np.abs(r[cand]) + self.bound[cand]) / self.n2[cand]
        w1[self.amb] += np.abs(r[self.amb]) / self.n2[self.amb]
        return w1, w2

    def check_h(self, h_g):
        assert self.h_sure <= h_g <= self.h_sure + self.n_amb, (h_g, self.h_sure, self.n_amb)

    def check_y(self, y_g, tol_rel):
        """Every element of y and its norm."""
        y_g = np.asarray(y_g, np.float64)
        assert y_g.shape == self.y.shape
        assert np.all(np.isfinite(y_g))
        err = np.abs(y_g - self.y)
        lim = tol_rel * np.abs(self.y) + self.B
        bad = np.nonzero(err > lim)[0]
        assert bad.size == 0, ("y differs beyond the bound at %d columns, first %d: gpu %r oracle %r "
                               "bound %r" % (bad.size, bad[0], y_g[bad[0]], self.y[bad[0]], lim[bad[0]]))
        assert np.linalg.norm(y_g - self.y) <= tol_rel * np.linalg.norm(self.y) + np.linalg.norm(self.B)

    def check_maxima(self, maxviol_g, maxb_g=None):
        tol_m = 4 * float(self.bound.max()) + 1e-12
        assert abs(maxviol_g - self.mr["maxviol"]) <= tol_m, (maxviol_g, self.mr["maxviol"], tol_m)
        if maxb_g is not None:
            assert abs(maxb_g - self.mr["maxb"]) <= 1e-6 * max(1.0, self.mr["maxb"])

    def step(self, h_g, lam, rule):
        """The oracle's step with the kernel's h (any h the classification
        allows) and its per-element bound."""
        if h_g == 0:
            return np.zeros_like(self.y), np.zeros_like(self.y)
        if rule == "relaxed":
            s = lam / h_g
            return s * self.y, s * self.B
        ny = np.linalg.norm(self.y)
        dny = np.linalg.norm(self.B)
        dx = lam * self.y / ny
        # |y_j/||y|| - y~_j/||y~||| <= (B_j + |y_j| ||B|| / ||y||) / (||y|| - ||B||)
        return dx, lam * (self.B + np.abs(self.y) * dny / ny) / max(ny - dny, 1e-300)


class MapRef(_Ref):
    """The oracle's Map/Reduce at (x, b) for a dense A with the
    classification of each row and the per-column bound B of the module
    docstring."""

    def __init__(self, A_eff, b, x, storage, depth, n2=None, levels=64, u=None):
        self.A = np.asarray(A_eff)
        if self.A.dtype not in (np.float32, np.float64):
            self.A = self.A.astype(np.float64)
        self.u = U[storage] if u is None else u
        Aabs = np.abs(self.A)
        if n2 is None:
            n2, _ = oracle.norms2(self.A)
        self.n2 = n2
        self.mr = oracle.map_reduce(self.A, b, n2, x)
        self.bound = residual_bound(self.A, x, b, self.u, levels, Aabs=Aabs)
        self._classify()
        keep = ~self.amb
        if keep.all():
            self.y = self.mr["y"]
        else:
            self.y = oracle.map_reduce(np.ascontiguousarray(self.A[keep]), np.asarray(b)[keep],
                                       n2[keep], x)["y"]
        w1, w2 = self._weights()
        self.B = _abs_matvec(Aabs.T, w1 + gamma(depth, self.u) * w2)


class CsrMapRef(_Ref):
    """The same for A in compressed rows (row_ptr, col_idx, val).  A row of
    L entries is summed over at most L + 16 levels (lanes, pieces of long
    rows, a warp tree); column j's y_j over its entries plus 16 levels."""

    def __init__(self, rp, ci, val, n, b, x, storage, n2=None, b_parts=None):
        rp = np.asarray(rp, np.int64)
        ci = np.asarray(ci)
        val = np.asarray(val, np.float64)
        self.u = u = U[storage]
        x = np.asarray(x, np.float64)
        b = np.asarray(b, np.float64)
        if n2 is None:
            n2, _ = oracle.norms2_csr(rp, val)
        self.n2 = n2
        self.mr = oracle.map_reduce_csr(rp, ci, val, n, b, n2, x)
        m = rp.size - 1
        L = np.diff(rp)
        row_of = np.repeat(np.arange(m), L)
        absdot = np.zeros(m)
        if val.size:
            absdot = np.bincount(row_of, weights=np.abs(val) * np.abs(x[ci]), minlength=m)
        # b_parts: the terms b is formed from (b0 and the tick shift), each
        # rounded to the accumulation type
        bsum = np.abs(b) if b_parts is None else sum(np.abs(t) for t in b_parts)
        g = np.array([gamma(int(l) + 16, u) for l in L]) if m < 200000 else \
            (L + 16) * u / (1 - (L.max() + 16) * u)
        self.bound = 2.0 * g * (absdot + bsum + 1e-300)
        self._classify()
        keep = np.flatnonzero(~self.amb)
        if keep.size == m:
            self.y = self.mr["y"]
        else:
            sub_rp = np.concatenate([[0], np.cumsum(L[keep])])
            sel = np.concatenate([np.arange(rp[i], rp[i + 1]) for i in keep]) if keep.size else \
                np.zeros(0, np.int64)
            self.y = oracle.map_reduce_csr(sub_rp, ci[sel], val[sel], n, b[keep], n2[keep], x)["y"]
        w1, w2 = self._weights()
        colcnt = np.bincount(ci, minlength=n) if ci.size else np.zeros(n, np.int64)
        gcol = (colcnt + 16) * u / (1 - (colcnt.max(initial=0) + 16) * u)
        av = np.abs(val)
        self.B = (np.bincount(ci, weights=av * w1[row_of], minlength=n) +
                  gcol * np.bincount(ci, weights=av * w2[row_of], minlength=n)) if ci.size else np.zeros(n)


def check_map_reduce(y_g, h_g, stats_g, A_eff, b, x, storage, depth, levels=64, n2=None, tol_rel=None):
    """One Map/Reduce of the CUDA path against the oracle at (x, b), element
    by element.  Returns the MapRef."""
    ref = MapRef(A_eff, b, to_accumulation(x, storage), storage, depth, n2=n2, levels=levels)
    ref.check_h(h_g)
    ref.check_y(y_g, TOL[storage] if tol_rel is None else tol_rel)
    if stats_g is not None:
        ref.check_maxima(stats_g["maxviol"], stats_g.get("maxb"))
    return ref


def implied_h(ref, dx_g, lam, rule):
    """The h of a relaxed step dx = lambda y / h, read off its largest
    element (None for ModAP, whose step does not involve h, and for a zero
    step).  A wrong classification or y shows up in the element checks."""
    if rule != "relaxed" or not np.any(ref.y):
        return None
    j = int(np.argmax(np.abs(ref.y)))
    if dx_g[j] == 0.0:
        return 0
    return int(round(lam * ref.y[j] / dx_g[j]))


def check_dx(ref, x_before, x_after, h_g, lam, rule, tol):
    """The step x_before - x_after of the CUDA path against ref's step, with
    the kernel's h (None: implied by the step), element by element and in
    norm."""
    x_before = np.asarray(x_before, np.float64)
    x_after = np.asarray(x_after, np.float64)
    dx_g = x_before - x_after        # x_{k+1} = x_k - dx
    if h_g is None:
        h_g = implied_h(ref, dx_g, lam, rule)
    if h_g is not None:
        ref.check_h(h_g)
    else:
        h_g = max(ref.h_sure, 1)     # ModAP: the step does not depend on h
    dx_ref, dB = ref.step(h_g, lam, rule)
    # the binary64 update x - s y and the subtraction here: a few units of x
    lim = tol * np.abs(dx_ref) + dB + 4 * 2.0 ** -53 * (np.abs(x_before) + np.abs(x_after))
    err = np.abs(dx_g - dx_ref)
    bad = np.nonzero(err > lim)[0]
    assert bad.size == 0, ("step differs beyond the bound at %d columns, first %d: gpu %r oracle %r "
                           "bound %r" % (bad.size, bad[0], dx_g[bad[0]], dx_ref[bad[0]], lim[bad[0]]))
    assert np.linalg.norm(dx_g - dx_ref) <= tol * np.linalg.norm(dx_ref) + \
        np.linalg.norm(lim - tol * np.abs(dx_ref))
    return ref


def check_step(x_before, x_after, h_g, A_eff, b, storage, depth, lam=1.0, rule="relaxed", n2=None,
               levels=64, tol_rel=None):
    """One iteration of the CUDA path from x_before (its own iterate) against
    the oracle's step from the same point, element by element."""
    tol = TOL[storage] if tol_rel is None else tol_rel
    ref = MapRef(A_eff, b, to_accumulation(x_before, storage), storage, depth, n2=n2, levels=levels)
    return check_dx(ref, x_before, x_after, h_g, lam, rule, tol)
