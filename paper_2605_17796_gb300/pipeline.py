"""Batched Monte-Carlo driver over the C ABI: sample -> decode (one or both sides) -> check.

All device buffers are torch tensors allocated once per chunk size; every step is one library
call enqueued on the current stream. Counting reductions (failures, iterations) run as torch
reductions on the device, so a chunk costs no host synchronisation until results are read.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import torch

from . import lead


@dataclass
class RunResult:
    shots: int = 0
    failures: int = 0
    logical: int = 0
    not_converged: int = 0
    iters_sum: int = 0
    per_side_failures: list = field(default_factory=lambda: [0, 0])


class Pipeline:
    """Preallocated buffers for `chunk` shots of one code on one device."""

    def __init__(self, code: lead.Code, chunk: int, device: int = 0):
        self.code = code
        self.chunk = int(chunk)
        self.device = torch.device("cuda", device)
        info = code.info
        kw = dict(device=self.device)
        self.err = [torch.zeros((chunk, info.words_n), dtype=torch.int32, **kw) for _ in range(2)]
        self.syn = [torch.zeros((chunk, info.words_m[s]), dtype=torch.int32, **kw) for s in range(2)]
        self.corr = [torch.zeros((chunk, info.words_n), dtype=torch.int32, **kw) for _ in range(2)]
        self.status = [torch.zeros(chunk, dtype=torch.uint8, **kw) for _ in range(2)]
        self.iters = [torch.zeros(chunk, dtype=torch.int32, **kw) for _ in range(2)]
        self.fail = [torch.zeros(chunk, dtype=torch.uint8, **kw) for _ in range(2)]
        ws = max(code.workspace_bytes(lead.opts(side=s, use_lead=True)) for s in range(2))
        self.workspace = torch.zeros(max(ws, 256) // 4 + 64, dtype=torch.int32, **kw)
        self._osd = None          # posterior / prior / workspace buffers, made on first OSD use
        self._iter = None         # posterior / workspace buffers of iterated LEAD, made on first use

    def _osd_buffers(self):
        if self._osd is None:
            info = self.code.info
            kw = dict(device=self.device)
            nb = max(self.code.osd_workspace_bytes(lead.opts(side=s), self.chunk) for s in range(2))
            self._osd = {"post": torch.zeros((self.chunk, info.n), dtype=torch.float32, **kw),
                         "prior": torch.zeros((self.chunk, info.n), dtype=torch.float32, **kw),
                         "ws": torch.zeros(nb // 4 + 64, dtype=torch.int32, **kw)}
        return self._osd

    def _iter_buffers(self):
        if self._iter is None:
            kw = dict(device=self.device)
            nb = max(self.code.iterated_workspace_bytes(lead.opts(side=s), self.chunk) for s in range(2))
            self._iter = {"post": torch.zeros((self.chunk, self.code.info.n), dtype=torch.float32, **kw),
                          "ws": torch.zeros(nb // 4 + 64, dtype=torch.int32, **kw)}
        return self._iter

    def sides_for(self, noise: int):
        return {lead.NOISE_X: [0], lead.NOISE_Z: [1], lead.NOISE_DEPOL: [0, 1]}[noise]

    def chunk_step(self, noise: int, p: float, shots: int, seed: int, offset: int, alpha: float = 1.0,
                   max_iter: int = 32, use_lead: bool = True, with_check: bool = True,
                   precision: int = lead.PREC_FP32, estimator: int = lead.EST_EXACT, osd_order=None,
                   rounds: int = 1):
        """One chunk (shots <= chunk): sample, decode the sides the noise touches (with OSD-CS of
        osd_order on the shots min-sum leaves unconverged, when given; with rounds > 1, iterated
        LEAD instead of one pass of Algorithm 1), check."""
        if rounds > 1 and osd_order is not None:
            raise ValueError("iterated LEAD and OSD post-processing are not combined")
        c = self.code
        sides = self.sides_for(noise)
        c.sample(noise, p, shots, seed, offset,
                 err_x=self.err[0] if 0 in sides else None, err_z=self.err[1] if 1 in sides else None,
                 syn_z=self.syn[0] if 0 in sides else None, syn_x=self.syn[1] if 1 in sides else None)
        p_side = p if noise != lead.NOISE_DEPOL else 2.0 * p / 3.0
        for s in sides:
            o = lead.opts(side=s, p=p_side, alpha=alpha, max_iter=max_iter, use_lead=use_lead, precision=precision,
                          estimator=estimator)
            if rounds > 1:
                b = self._iter_buffers()
                c.decode_iterated(o, rounds, self.syn[s], shots, self.corr[s], self.status[s], self.iters[s],
                                  llr=b["post"][:shots], workspace=b["ws"])
            elif osd_order is None:
                c.decode(o, self.syn[s], shots, self.corr[s], self.status[s], self.iters[s],
                         workspace=self.workspace)
            else:
                b = self._osd_buffers()
                post, prior = b["post"][:shots], None
                c.decode(o, self.syn[s], shots, self.corr[s], self.status[s], self.iters[s], llr=post,
                         workspace=self.workspace)
                if use_lead:
                    prior = b["prior"][:shots]
                    po = lead.opts(side=s, p=p_side, alpha=alpha, estimator=estimator)
                    c.local_estimate(po, self.syn[s], shots, prior, self.workspace)
                c.osd(o, osd_order, self.syn[s], shots, post, self.status[s], self.corr[s], prior=prior,
                      workspace=b["ws"])
            if with_check:
                c.check(s, self.err[s], self.corr[s], shots, self.fail[s])
        return sides

    def run(self, noise: int, p: float, shots: int, seed: int = 0, offset: int = 0, alpha: float = 1.0,
            max_iter: int = 32, use_lead: bool = True, precision: int = lead.PREC_FP32,
            estimator: int = lead.EST_EXACT, osd_order=None, rounds: int = 1) -> RunResult:
        """Decode `shots` shots in chunks and return failure / iteration counts."""
        acc = None
        done = 0
        while done < shots:
            n = min(self.chunk, shots - done)
            sides = self.chunk_step(noise, p, n, seed, offset + done, alpha, max_iter, use_lead,
                                    precision=precision, estimator=estimator, osd_order=osd_order,
                                    rounds=rounds)
            fail_any = torch.zeros(n, dtype=torch.bool, device=self.device)
            logical = torch.zeros(n, dtype=torch.bool, device=self.device)
            nc = torch.zeros(n, dtype=torch.bool, device=self.device)
            its = torch.zeros((), dtype=torch.int64, device=self.device)
            side_f = []
            for s in sides:
                f = self.fail[s][:n]
                fail_any |= f != 0
                logical |= (f & 2) != 0
                nc |= (self.status[s][:n] & lead.ST_MAX_ITER) != 0
                its = its + self.iters[s][:n].sum()
                side_f.append((f != 0).sum())
            vec = torch.stack([fail_any.sum(), logical.sum(), nc.sum(), its] +
                              [side_f[i] if i < len(side_f) else torch.zeros((), dtype=torch.int64,
                                                                             device=self.device)
                               for i in range(2)])
            acc = vec if acc is None else acc + vec
            done += n
        v = acc.tolist()
        r = RunResult(shots=shots, failures=int(v[0]), logical=int(v[1]), not_converged=int(v[2]),
                      iters_sum=int(v[3]))
        sides = self.sides_for(noise)
        r.per_side_failures = [0, 0]
        for i, s in enumerate(sides):
            r.per_side_failures[s] = int(v[4 + i])
        return r
