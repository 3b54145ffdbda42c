"""Batched backward Riccati recursion over MPC instances of uneven sizes.

Marshalling for bf_driccati_sqrt_batched (include/bfgpu.h): RiccatiBatch lays
out every instance's panel-major matrices in one device tensor, builds the
device array of bf_riccati_prob descriptors, orders the instances by
decreasing cost and splits them into size buckets, one launch per bucket
(each launch sizes its shared memory for its bucket).  An autotuner picks
the CTA width of each bucket by timing the candidates on the actual batch.
All arithmetic runs in the CUDA library.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _abi, _check, _stream, _torch, load

# instance buckets by m = nx + nu (upper bounds); one launch per non-empty bucket
BUCKETS = (24, 40, 56, 80, 128)


def stage_flops(nx: int, nu: int) -> float:
    """Flops of one stage: trmm m*nx(nx+1), syrk nx*m(m+1), potrf m^3/3+m^2/2+m/6, trsm nx*nu^2."""
    m = nx + nu
    return m * nx * (nx + 1) + nx * m * (m + 1) + m ** 3 / 3.0 + m ** 2 / 2.0 + m / 6.0 + nx * nu * nu


def _pm(r):
    return -(-r // _abi.BF_PS) * _abi.BF_PS


class RiccatiBatch:
    def __init__(self, nx, nu, N: int, device=None):
        torch = _torch()
        self.nx = np.asarray(nx, dtype=np.int64)
        self.nu = np.asarray(nu, dtype=np.int64)
        self.batch = len(self.nx)
        self.N = int(N)
        self.device = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        # group instances of equal shape so that each group packs in one call
        shapes = sorted({(int(a), int(b)) for a, b in zip(self.nx, self.nu)})
        self.groups = []  # (nx, nu, instance indices, first double offset, region doubles)
        off = 0
        self.region = np.zeros(self.batch, dtype=np.int64)
        self.offset = np.zeros(self.batch, dtype=np.int64)
        for (a, b) in shapes:
            idx = np.nonzero((self.nx == a) & (self.nu == b))[0]
            m = a + b
            sizes = [_pm(m) * a, _pm(m) * m, _pm(a) * a, self.N * _pm(a) * a, self.N * _pm(a) * b]
            reg = sum((s + 3) // 4 * 4 for s in sizes)
            self.groups.append((a, b, idx, off, reg, sizes))
            self.offset[idx] = off + reg * np.arange(len(idx))
            self.region[idx] = reg
            off += reg * len(idx)
        self.total = off
        self.buf = torch.zeros(max(1, off), dtype=torch.float64, device=self.device)
        self.info = torch.zeros(self.batch * self.N, dtype=torch.int32, device=self.device)
        base = self.buf.data_ptr()
        descs = (_abi.bf_riccati_prob * self.batch)()
        for (a, b, idx, off0, reg, sizes) in self.groups:
            offs = np.cumsum([0] + [(s + 3) // 4 * 4 for s in sizes[:-1]])
            for q, i in enumerate(idx):
                o = base + 8 * (off0 + reg * q)
                d = descs[i]
                d.nx, d.nu = a, b
                d.BAt, d.bat_cn = o + 8 * int(offs[0]), a
                d.M0, d.m0_cn = o + 8 * int(offs[1]), a + b
                d.LN, d.ln_cn = o + 8 * int(offs[2]), a
                d.L, d.l_cn, d.l_stride = o + 8 * int(offs[3]), a, _pm(a) * a
                d.Kt, d.kt_cn, d.kt_stride = o + 8 * int(offs[4]), b, _pm(a) * b
                d.info = self.info.data_ptr() + 4 * self.N * int(i)
        raw = bytes(descs)
        self.probs = torch.frombuffer(bytearray(raw), dtype=torch.uint8).to(self.device)
        self._offs = {g[0:2]: np.cumsum([0] + [(s + 3) // 4 * 4 for s in g[5][:-1]]) for g in self.groups}
        # decreasing-cost order, split into buckets by m
        cost = np.array([stage_flops(a, b) for a, b in zip(self.nx, self.nu)])
        self.flops = float(cost.sum()) * self.N
        m = self.nx + self.nu
        self.buckets = []  # (indices tensor, max_nx, max_nu, threads)
        lo = 0
        for hi in BUCKETS + (10 ** 9,):
            sel = np.nonzero((m > lo) & (m <= hi))[0]
            lo = hi
            if len(sel) == 0:
                continue
            sel = sel[np.argsort(-cost[sel], kind="stable")]
            t = torch.from_numpy(sel.astype(np.int32)).to(self.device)
            self.buckets.append([t, int(self.nx[sel].max()), int(self.nu[sel].max()), 0])

    # ---- data movement (pack / unpack through the library) ---------------

    def _mat_desc(self, g, which, rows, cols):
        """Descriptor of matrix `which` (0 BAt, 1 M0, 2 LN, 3 L, 4 Kt) of group g's first instance."""
        a, b, idx, off0, reg, sizes = g
        d = _abi.bf_dmat()
        d.pA = self.buf.data_ptr() + 8 * (off0 + int(self._offs[(a, b)][which]))
        d.dA = None
        d.m, d.n, d.pm, d.cn, d.ps = rows, cols, _pm(rows), cols, _abi.BF_PS
        d.memsize = 0
        return d

    def _pack_group(self, g, which, X, rows, cols):
        """X: (count, rows, cols) tensor -> panel-major matrix `which` of each instance of group g."""
        torch = _torch()
        cm = X.to(self.device, torch.float64).transpose(1, 2).contiguous()
        d = self._mat_desc(g, which, rows, cols)
        _check("bf_pack_dmat_batched", load().bf_pack_dmat_batched(
            len(g[2]), rows, cols, ctypes.c_void_p(cm.data_ptr()), rows, rows * cols, ctypes.byref(d), 0, 0,
            g[4], _stream()))
        torch.cuda.current_stream().synchronize()

    def set_inputs(self, A, B, M0=None, LN=None):
        """A[i] (nx x nx), B[i] (nx x nu): lists of tensors per instance, or a callable
        (nx, nu, count) -> (A, B) batch per shape group.  M0 defaults to I
        (Q = R = I, S = 0) and LN to I (P_N = I)."""
        torch = _torch()
        for g in self.groups:
            a, b, idx = g[0], g[1], g[2]
            if callable(A):
                Ag, Bg = A(a, b, len(idx))
            else:
                Ag = torch.stack([torch.as_tensor(A[i]) for i in idx])
                Bg = torch.stack([torch.as_tensor(B[i]) for i in idx])
            BAt = torch.cat([Bg.transpose(1, 2), Ag.transpose(1, 2)], dim=1)  # (count, nu+nx, nx)
            self._pack_group(g, 0, BAt, a + b, a)
            if M0 is None:
                M = torch.eye(a + b, dtype=torch.float64).expand(len(idx), a + b, a + b)
            else:
                M = torch.stack([torch.as_tensor(M0[i]) for i in idx])
            self._pack_group(g, 1, M, a + b, a + b)
            if LN is None:
                Ln = torch.eye(a, dtype=torch.float64).expand(len(idx), a, a)
            else:
                Ln = torch.stack([torch.as_tensor(LN[i]) for i in idx])
            self._pack_group(g, 2, Ln, a, a)

    def _unpack(self, i, which, rows, cols, k):
        torch = _torch()
        a, b = int(self.nx[i]), int(self.nu[i])
        g = next(g for g in self.groups if g[0] == a and g[1] == b)
        q = int(np.nonzero(g[2] == i)[0][0])
        d = self._mat_desc(g, which, rows, cols)
        stride = _pm(a) * (a if which == 3 else b)
        d.pA = d.pA + 8 * (g[4] * q + stride * k)
        out = torch.empty(1, cols, rows, dtype=torch.float64, device=self.device)
        _check("bf_unpack_dmat_batched", load().bf_unpack_dmat_batched(
            1, rows, cols, ctypes.byref(d), 0, 0, 0, ctypes.c_void_p(out.data_ptr()), rows, rows * cols,
            _stream()))
        torch.cuda.current_stream().synchronize()
        return out[0].transpose(0, 1).cpu().numpy()

    def factor(self, i, k):
        """L_k of instance i (lower triangle; zeros above)."""
        a = int(self.nx[i])
        return np.tril(self._unpack(i, 3, a, a, k))

    def gain_t(self, i, k):
        """Kt_k = K_k^T of instance i (nx x nu)."""
        return self._unpack(i, 4, int(self.nx[i]), int(self.nu[i]), k)

    def infos(self):
        return self.info.view(self.batch, self.N).cpu().numpy()

    # ---- launch -------------------------------------------------------------

    def run(self, stream=None):
        lib = load()
        s = _stream(stream)
        for (idx, mnx, mnu, thr) in self.buckets:
            _check("bf_driccati_sqrt_batched", lib.bf_driccati_sqrt_batched(
                len(idx), self.N, ctypes.c_void_p(self.probs.data_ptr()), ctypes.c_void_p(idx.data_ptr()),
                mnx, mnu, thr, s))

    def autotune(self, candidates=(64, 128, 256, 512), reps=2):
        """Pick each bucket's CTA width by timing the candidates on this batch."""
        torch = _torch()
        lib = load()
        s = _stream()
        choice = []
        for bk in self.buckets:
            idx, mnx, mnu, _ = bk
            best = None
            for thr in candidates:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                _check("riccati", lib.bf_driccati_sqrt_batched(len(idx), self.N, ctypes.c_void_p(self.probs.data_ptr()),
                                                               ctypes.c_void_p(idx.data_ptr()), mnx, mnu, thr, s))
                e0.record()
                for _ in range(reps):
                    lib.bf_driccati_sqrt_batched(len(idx), self.N, ctypes.c_void_p(self.probs.data_ptr()),
                                                 ctypes.c_void_p(idx.data_ptr()), mnx, mnu, thr, s)
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / reps
                if best is None or ms < best[1]:
                    best = (thr, ms)
            bk[3] = best[0]
            choice.append({"max_m": mnx + mnu, "instances": len(idx), "threads": best[0], "ms": round(best[1], 4)})
        return choice
