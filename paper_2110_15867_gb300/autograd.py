"""Reverse mode of a run of Eq. (5) steps as a ``torch.autograd.Function``.

``VlasovRun.apply(f0, phi, run, dt, a_half, n_steps, K)`` advances ``f0`` by
``n_steps`` steps with the external potential ``phi`` (both kicks use phi, the
drift uses ``a_half``) and returns the density rho_nu(x) (FP64) of the final state.
Its backward gives dL/df0 and dL/dphi for any loss of rho_nu.

Memory: the forward keeps the state every K steps (checkpoints) and runs the trailing
segments that the tape holds with ``vlasov_step_record``, which keeps the input of every
sweep (each sweep writes the next record, so recording costs no copies).  The backward
takes the segments last to first: a taped one is already recorded; each other one is run
again from its checkpoint with ``vlasov_step_record``; then ``vlasov_step_adjoint_recorded``
is applied step by step in reverse.  Each taped segment holds 8 K + K - 1 arrays the size
of f; the tape is reused by later calls.  How many segments are taped is
``run.tape_segments``: a number, or "auto" (the default): as many as fit in half the
device memory that is free (or held by the tape) when the forward starts, at least one.
With every segment taped the backward runs no forward step again.

Every operation on f or lambda runs in libvlasov's kernels through the C ABI; this
module only orders the calls and owns the buffers.
"""
from __future__ import annotations

import torch

from .binding import Vlasov


class Run:
    """A context and the buffers of one grid: the working state and the tape.

    tape_segments: how many trailing checkpoint segments the forward records directly
    (each holds 8 K + K - 1 arrays the size of f); the backward runs the other segments
    again.  More segments trade memory for less recomputation.  "auto": as many as fit in
    tape_budget bytes (default: half the device memory free, or already held by the tape,
    when a forward starts), at least one."""

    def __init__(self, shape, dtype=torch.float32, device="cuda", L: float = 1.0, V: float = 5.0,
                 tape_segments="auto", tape_budget=None):
        if tape_segments != "auto" and int(tape_segments) < 1:
            raise ValueError("tape_segments must be >= 1 or 'auto'")
        self.shape = tuple(shape)
        self.work = torch.empty(self.shape, dtype=dtype, device=device)
        self.v = Vlasov(self.work, L=L, V=V)
        self.tape_segments = tape_segments
        self.tape_budget = tape_budget
        self._slots = []
        self.tape_owner = None  # the forward whose trailing segments the tape holds

    def taped_segments(self, nseg: int, K: int) -> int:
        """Trailing segments of a run of nseg segments of K steps that the forward records."""
        if self.tape_segments != "auto":
            return max(1, min(nseg, int(self.tape_segments)))
        seg_bytes = (9 * K - 1) * self.work.numel() * self.work.element_size()
        held = sum(t.numel() * t.element_size() for rec, states in self._slots for r in rec for t in r) + \
            sum(t.numel() * t.element_size() for rec, states in self._slots for t in states)
        if self.tape_budget is not None:
            budget = float(self.tape_budget)
        else:
            budget = 0.5 * (torch.cuda.mem_get_info(self.work.device)[0] + held)
        return max(1, min(nseg, int(budget // seg_bytes)))

    def slot(self, i: int, K: int):
        """Tape slot i: records for K steps (8 arrays each) and K - 1 intermediate states."""
        while len(self._slots) <= i:
            self._slots.append(([], []))
        rec, states = self._slots[i]
        while len(rec) < K:
            rec.append([torch.empty_like(self.work) for _ in range(8)])
        while len(states) < K - 1:
            states.append(torch.empty_like(self.work))
        return rec, states

    def tape(self, K: int):
        return self.slot(0, K)

    def release_tape(self):
        self._slots = []

    def close(self):
        self.release_tape()
        self.v.close()


class VlasovRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f0, phi, run: Run, dt: float, a_half: float, n_steps: int, K: int = 4):
        if K < 1 or n_steps < 1:
            raise ValueError("need n_steps >= 1 and K >= 1")
        phi32 = phi.detach().to(torch.float32).contiguous()
        v = run.v
        nseg = (n_steps + K - 1) // K
        first_taped = max(0, nseg - run.taped_segments(nseg, K))
        run.work.copy_(f0.detach())
        starts = [f0.detach().contiguous()]  # the state at the start of every segment
        for n in range(first_taped * K):
            if n > 0 and n % K == 0:
                starts.append(run.work.clone())
            v.step(dt, a_half, a_half, phi32)
        if first_taped > 0:
            starts.append(run.work.clone())
        # the trailing segments, recorded: each one's final state starts the next; the last lands in run.work
        for sgi in range(first_taped, nseg):
            m = min(K, n_steps - sgi * K)
            rec, states = run.slot(sgi - first_taped, K)
            last_seg = sgi == nseg - 1
            end = run.work if last_seg else torch.empty_like(run.work)
            seq = [starts[sgi]] + states[:m - 1] + [end]
            for i in range(m):
                v.step_record(seq[i], rec[i], dt, a_half, phi32, f_next=seq[i + 1])
            if not last_seg:
                starts.append(end)
        token = object()
        run.tape_owner = token
        rho = v.moment()
        ctx.save_for_backward(f0, phi)
        ctx.starts, ctx.first_taped = starts[1:], first_taped
        ctx.token = token
        ctx.run, ctx.dt, ctx.a_half, ctx.n_steps, ctx.K = run, dt, a_half, n_steps, K
        return rho

    @staticmethod
    def backward(ctx, grad_rho):
        f0, phi = ctx.saved_tensors
        run, dt, a_half, n_steps, K = ctx.run, ctx.dt, ctx.a_half, ctx.n_steps, ctx.K
        v = run.v
        phi32 = phi.detach().to(torch.float32).contiguous()
        lam = torch.empty_like(run.work)
        v.moment_adjoint(grad_rho.detach().to(torch.float64).contiguous(), lam)
        dphi = torch.zeros(phi32.shape, dtype=torch.float64, device=phi32.device)
        starts = [f0.detach().contiguous()] + ctx.starts
        taped = run.tape_owner is ctx.token  # no other forward has reused the tape since
        for s in reversed(range(len(starts))):
            m = min(K, n_steps - s * K)
            on_tape = taped and s >= ctx.first_taped
            rec, states = run.slot(s - ctx.first_taped if on_tape else 0, K)
            seq = [starts[s]] + states[:m - 1]
            if not on_tape:
                for i in range(m):
                    v.step_record(seq[i], rec[i], dt, a_half, phi32, f_next=seq[i + 1] if i + 1 < m else None)
            for i in reversed(range(m)):
                v.step_adjoint_recorded(seq[i], rec[i], lam, dt, a_half, phi32, dphi)
            if on_tape and s == ctx.first_taped:
                taped = False  # the slots are reused from here on
        run.tape_owner = None
        ctx.starts = None
        return lam, dphi.to(phi.dtype), None, None, None, None, None


def _sched(x, n):
    return [float(x)] * n if isinstance(x, (int, float)) else [float(v) for v in x]


class VlasovRunSC(torch.autograd.Function):
    """rho_nu after n self-consistent steps (Eq. 5 with phi^{n+1} from the post-drift moment
    plus rho_bg): the state is (f, phi).  Inputs f0, phi0 (FP32) and rho_bg (FP64, may be
    None); a_half / a_full: one value or one per step.  Checkpoints (f, phi) every K steps;
    the backward chains dL/dphi^{n+1} from step to step through
    ``vlasov_step_adjoint_recorded_sc`` and returns dL/df0, dL/dphi0, dL/drho_bg."""

    @staticmethod
    def forward(ctx, f0, phi0, rho_bg, run: Run, dt: float, a_half, a_full, n_steps: int, K: int = 4,
                four_pi_G: float = 1.0):
        if K < 1 or n_steps < 1:
            raise ValueError("need n_steps >= 1 and K >= 1")
        ah, af = _sched(a_half, n_steps), _sched(a_full, n_steps)
        v = run.v
        bg = None if rho_bg is None else rho_bg.detach().to(torch.float64).contiguous()
        phi = phi0.detach().to(torch.float32).contiguous()
        run.work.copy_(f0.detach())
        nseg = (n_steps + K - 1) // K
        first_taped = max(0, nseg - run.taped_segments(nseg, K))
        starts = [(f0.detach().contiguous(), phi)]  # (f, phi) at the start of every segment
        for n in range(first_taped * K):
            if n > 0 and n % K == 0:
                starts.append((run.work.clone(), phi))
            phi_next = torch.empty_like(phi)
            v.step(dt, ah[n], af[n], phi, rho_bg=bg, four_pi_G=four_pi_G, phi_next=phi_next)
            phi = phi_next
        if first_taped > 0:
            starts.append((run.work.clone(), phi))
        # the trailing segments, recorded with the potential of every step
        taped_phis = []
        for sgi in range(first_taped, nseg):
            m = min(K, n_steps - sgi * K)
            rec, states = run.slot(sgi - first_taped, K)
            last_seg = sgi == nseg - 1
            end = run.work if last_seg else torch.empty_like(run.work)
            seq = [starts[sgi][0]] + states[:m - 1] + [end]
            phis = [starts[sgi][1]] + [torch.empty_like(phi) for _ in range(m)]
            for i in range(m):
                n = sgi * K + i
                v.step_record_sc(seq[i], rec[i], dt, ah[n], af[n], phis[i], phis[i + 1], rho_bg=bg,
                                 four_pi_G=four_pi_G, f_next=seq[i + 1])
            taped_phis.append(phis)
            if not last_seg:
                starts.append((end, phis[m]))
        token = object()
        run.tape_owner = token
        rho = v.moment()
        ctx.save_for_backward(f0, phi0)
        ctx.bg, ctx.starts, ctx.taped_phis, ctx.first_taped, ctx.token = bg, starts, taped_phis, first_taped, token
        ctx.has_bg = rho_bg is not None
        ctx.run, ctx.dt, ctx.ah, ctx.af, ctx.n_steps, ctx.K, ctx.G = run, dt, ah, af, n_steps, K, four_pi_G
        return rho

    @staticmethod
    def backward(ctx, grad_rho):
        f0, phi0 = ctx.saved_tensors
        run, dt, ah, af, n_steps, K, G = ctx.run, ctx.dt, ctx.ah, ctx.af, ctx.n_steps, ctx.K, ctx.G
        v = run.v
        shape3 = tuple(phi0.shape)
        lam = torch.empty_like(run.work)
        v.moment_adjoint(grad_rho.detach().to(torch.float64).contiguous(), lam)
        lam_phi = None
        dbg = torch.zeros(shape3, dtype=torch.float64, device=lam.device) if ctx.has_bg else None
        starts = ctx.starts
        taped = run.tape_owner is ctx.token  # no other forward has reused the tape since
        for s in reversed(range(len(starts))):
            m = min(K, n_steps - s * K)
            on_tape = taped and s >= ctx.first_taped
            rec, states = run.slot(s - ctx.first_taped if on_tape else 0, K)
            seq = [starts[s][0]] + states[:m - 1]
            if on_tape:
                phis = ctx.taped_phis[s - ctx.first_taped]
            else:
                phis = [starts[s][1]] + [torch.empty_like(starts[s][1]) for _ in range(m)]
                for i in range(m):
                    v.step_record_sc(seq[i], rec[i], dt, ah[s * K + i], af[s * K + i], phis[i], phis[i + 1],
                                     rho_bg=ctx.bg, four_pi_G=G, f_next=seq[i + 1] if i + 1 < m else None)
            for i in reversed(range(m)):
                dphi = torch.zeros(shape3, dtype=torch.float64, device=lam.device)
                v.step_adjoint_recorded_sc(seq[i], rec[i], lam, dt, ah[s * K + i], af[s * K + i], phis[i],
                                           phis[i + 1], G, lam_phi_next=lam_phi, dLdphi_n=dphi, dLdrho_bg=dbg)
                lam_phi = dphi
            if on_tape and s == ctx.first_taped:
                taped = False  # the slots are reused from here on
        run.tape_owner = None
        ctx.starts = ctx.taped_phis = None
        dphi0 = lam_phi.to(phi0.dtype) if lam_phi is not None else None
        return lam, dphi0, dbg, None, None, None, None, None, None, None


def run_rho_sc(f0, phi0, rho_bg, run: Run, dt: float, a_half, a_full, n_steps: int, K: int = 4,
               four_pi_G: float = 1.0):
    """rho_nu after n_steps self-consistent steps from (f0, phi0), differentiable in f0, phi0
    and rho_bg."""
    return VlasovRunSC.apply(f0, phi0, rho_bg, run, dt, a_half, a_full, n_steps, K, four_pi_G)


def run_rho(f0, phi, run: Run, dt: float, a_half: float, n_steps: int, K: int = 4):
    """rho_nu after n_steps steps from f0 under phi, differentiable in f0 and phi."""
    return VlasovRun.apply(f0, phi, run, dt, a_half, n_steps, K)
