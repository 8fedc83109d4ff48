"""Python face of libtufrg: one ``Model`` per lattice model, device buffers as torch tensors.

Every numerical step runs in the library's CUDA kernels; this module only
marshals arguments (descriptor arrays, device pointers, the current torch
stream) and turns status codes into exceptions.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional

import numpy as np
import torch

from . import _lib
from ._lib import (BASIS_BAND, BASIS_ORBITAL, CH_C, CH_P, FP64, LOOPS_AUTO, LOOPS_SIMT, LOOPS_TC, PRODUCTS_AUTO, PRODUCTS_SIMT, PRODUCTS_TC, SPLIT32, SYMMETRIC_STATE, SYMMETRY_AUTO,
                   SYMMETRY_OFF, SYMMETRY_STATES,
                   FlowOpts, FlowResult, FlowStepInfo, ModelDesc, TufrgError)
from .inputs import FLOW_ATOL, FLOW_RTOL, FLOW_STOP, FLOW_T0, FLOW_T_END, ModelSpec

__all__ = ["Model", "flow_batch", "FP64", "SPLIT32", "PRODUCTS_AUTO", "PRODUCTS_TC", "PRODUCTS_SIMT", "SYMMETRY_AUTO",
           "SYMMETRY_OFF", "SYMMETRY_STATES", "SYMMETRIC_STATE", "CH_P", "CH_C", "LOOPS_AUTO", "LOOPS_TC", "LOOPS_SIMT",
           "BASIS_ORBITAL", "BASIS_BAND", "TufrgError"]


def _ptr(t) -> int:
    return t.data_ptr() if isinstance(t, torch.Tensor) else t.ctypes.data


class Model:
    """A TU-fRG model on the current CUDA device (see include/tufrg.h for layouts)."""

    def __init__(self, spec: ModelSpec, precision: int = FP64, stream: Optional[torch.cuda.Stream] = None,
                 mu: Optional[float] = None, products: int = PRODUCTS_AUTO, symmetry: int = SYMMETRY_AUTO,
                 loops: int = LOOPS_AUTO, basis: int = BASIS_ORBITAL):
        if not torch.cuda.is_available():
            raise RuntimeError("libtufrg needs a CUDA device")
        self.spec = spec
        self.precision = precision
        self.basis = basis
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._L = _lib.lib()
        # keep the descriptor arrays alive for the duration of the init call
        self._hopR = np.ascontiguousarray(spec.hop_R, np.int32)
        self._hopt = np.ascontiguousarray(spec.hop_t, np.complex128)
        self._V0 = np.ascontiguousarray(spec.V0, np.complex128)
        self._ffR = np.ascontiguousarray(spec.ff_R, np.int32)
        use_fill = mu is None and spec.filling > 0
        d = ModelDesc(spec.n_s, self._hopR.shape[0], self._hopR.ctypes.data, self._hopt.ctypes.data,
                      float(spec.mu if mu is None else mu), float(spec.filling if use_fill else 0.0),
                      float(spec.T_mu), self._V0.ctypes.data, self._ffR.shape[0], self._ffR.ctypes.data,
                      spec.Lq, spec.nc, int(precision), int(products), int(symmetry),
                      int(getattr(spec, "regulator", 0)), float(getattr(spec, "T_reg", 0.05)), int(loops), int(basis))
        h = C.c_void_p()
        st = self._L.tufrg_init_model(C.byref(d), C.c_void_p(self.stream.cuda_stream), C.byref(h))
        self._h = h
        if st != 0:
            msg = self._L.tufrg_last_error(h).decode() if h.value else ""
            self._L.tufrg_free(h)
            self._h = C.c_void_p()
            raise TufrgError(st, msg)
        Nq, M, nd, Nk = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        mu_ = C.c_double()
        self._check(self._L.tufrg_dims(self._h, C.byref(Nq), C.byref(M), C.byref(nd), C.byref(Nk), C.byref(mu_)))
        self.Nq, self.M, self.nd, self.Nk, self.mu = Nq.value, M.value, nd.value, Nk.value, mu_.value
        dl = np.zeros((self.nd, 2), np.int32)
        self._check(self._L.tufrg_deltas(self._h, dl.ctypes.data))
        self.deltas = dl
        pr, t_tc, t_simt = C.c_int(), C.c_double(), C.c_double()
        self._check(self._L.tufrg_model_info(self._h, C.byref(pr), C.byref(t_tc), C.byref(t_simt)))
        self.products = {PRODUCTS_TC: "tc", PRODUCTS_SIMT: "simt"}.get(pr.value, "?")
        self.products_tuning_ms = {"tc": t_tc.value, "simt": t_simt.value}
        nl = C.c_int()
        self._check(self._L.tufrg_loop_momenta(self._h, C.byref(nl)))
        self.n_loop_q = nl.value   # transfer momenta whose loop k-sums run directly
        lb = C.c_int()
        self._check(self._L.tufrg_loops_info(self._h, C.byref(lb)))
        self.loops_backend = {LOOPS_TC: "tc", LOOPS_SIMT: "simt"}.get(lb.value, "?")
        kyc, ncand = C.c_int(), C.c_int()
        cand_ms = np.zeros(16)
        self._check(self._L.tufrg_loop_tiles(self._h, C.byref(kyc), C.byref(ncand), cand_ms.ctypes.data, len(cand_ms)))
        # the loop k-sum's ky ranges per column, and the timed candidates {ranges: ms per launch} when tuned
        self.loop_ky_chunks = kyc.value
        self.loop_tiles_tuning_ms = {c + 1: float(cand_ms[c]) for c in range(min(ncand.value, len(cand_ms)))}
        tw, ntc = C.c_int(), C.c_int()
        tc_ms = np.zeros(4)
        self._check(self._L.tufrg_products_tiles(self._h, C.byref(tw), C.byref(ntc), tc_ms.ctypes.data, len(tc_ms)))
        # the tensor-core products' tile width (complex columns) and the autotuner's timings of its candidates
        self.products_tile_width = tw.value
        self.products_tiles_tuning_ms = [float(tc_ms[c]) for c in range(min(ntc.value, len(tc_ms)))]
        su, t_gen, t_rep = C.c_int(), C.c_double(), C.c_double()
        self._check(self._L.tufrg_symmetry_info(self._h, C.byref(su), C.byref(t_gen), C.byref(t_rep)))
        self.symmetric_state_path = bool(su.value)   # rhs(symmetric=True) works at the representatives only
        self.symmetric_state_tuning_ms = {"general": t_gen.value, "representatives": t_rep.value}

    # ------------------------------------------------------------------ plumbing
    def _check(self, st: int):
        if st != 0:
            raise TufrgError(st, self._L.tufrg_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._L.tufrg_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def device(self):
        return torch.device("cuda", torch.cuda.current_device())

    def state_shape(self):
        return (2, self.Nq, self.M, self.M)

    def loop_shape(self):
        ns2 = self.spec.n_s ** 2
        return (2, self.Nq, self.nd, ns2, ns2)

    def zeros_state(self) -> torch.Tensor:
        return torch.zeros(self.state_shape(), dtype=torch.complex128, device=self.device)

    def _dev(self, x) -> torch.Tensor:
        if isinstance(x, np.ndarray):
            x = torch.from_numpy(np.ascontiguousarray(x, np.complex128))
        x = x.to(device=self.device, dtype=torch.complex128)
        return x.contiguous()

    # ------------------------------------------------------------------ entry points
    def gather_table(self, channel: int) -> np.ndarray:
        n = C.c_int()
        self._check(self._L.tufrg_gather_table(self._h, channel, None, 0, C.byref(n)))
        out = np.zeros((n.value, 9), np.int32)
        self._check(self._L.tufrg_gather_table(self._h, channel, out.ctypes.data, n.value, C.byref(n)))
        return out

    def bands(self):
        E = torch.empty((self.Nk, self.spec.n_s), dtype=torch.float64, device=self.device)
        U = torch.empty((self.Nk, self.spec.n_s, self.spec.n_s), dtype=torch.complex128, device=self.device)
        self._check(self._L.tufrg_bands(self._h, _ptr(E), _ptr(U)))
        return E, U

    def loops(self, T: float, mask: int = CH_P | CH_C, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        if out is None:
            out = torch.zeros(self.loop_shape(), dtype=torch.complex128, device=self.device)
        self._check(self._L.tufrg_loops(self._h, float(T), int(mask), _ptr(out)))
        return out

    def project(self, state, mask: int = CH_P | CH_C, out: Optional[torch.Tensor] = None, want_max: bool = True):
        state = self._dev(state)
        if out is None:
            out = torch.empty_like(state)
        amax = C.c_double(0.0)
        self._check(self._L.tufrg_project(self._h, _ptr(state), int(mask), _ptr(out),
                                          C.byref(amax) if want_max else None))
        return out, amax.value

    def rhs(self, T: float, state, mask: int = CH_P | CH_C, out: Optional[torch.Tensor] = None,
            symmetric: bool = False) -> torch.Tensor:
        """dX/dT at T.  symmetric=True asserts that the state has the model's loop symmetries (every state of a
        flow from X = 0 does): projections and products then run for the orbit representatives only."""
        state = self._dev(state)
        if out is None:
            out = torch.empty_like(state)
        flag = SYMMETRIC_STATE if symmetric else 0
        self._check(self._L.tufrg_rhs(self._h, float(T), _ptr(state), int(mask) | flag, _ptr(out)))
        return out

    def rhs_host(self, T: float, state_host: torch.Tensor, out_host: torch.Tensor, mask: int = CH_P | CH_C):
        """dX/dT with host (ideally pinned) buffers: H2D, evaluation and D2H inside the call."""
        if state_host.device.type != "cpu" or out_host.device.type != "cpu":
            raise ValueError("rhs_host takes host tensors")
        if not (state_host.is_contiguous() and out_host.is_contiguous()):
            raise ValueError("rhs_host needs C-contiguous host tensors")
        if state_host.dtype != torch.complex128 or out_host.dtype != torch.complex128:
            raise ValueError("rhs_host needs complex128 tensors")
        if tuple(state_host.shape) != self.state_shape() or tuple(out_host.shape) != self.state_shape():
            raise ValueError(f"rhs_host needs tensors of shape {self.state_shape()}")
        self._check(self._L.tufrg_rhs_host(self._h, float(T), _ptr(state_host), int(mask), _ptr(out_host)))
        return out_host

    def band_basis(self, state, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """The exchange propagators P, C of ``state`` in the band basis of the model's eigenvectors (``bands()``),
        two-band models (Sec. 3.4, Eqs. mat_trafo_P, mat_trafo_D)."""
        state = self._dev(state)
        if out is None:
            out = torch.empty_like(state)
        self._check(self._L.tufrg_band_basis(self._h, _ptr(state), _ptr(out)))
        return out

    def rhs_host_batch(self, T, states_host, outs_host, mask: int = CH_P | CH_C, symmetric: bool = False):
        """dX/dT for a sequence of host (ideally pinned) states, the transfers of neighbouring steps overlapped with
        the evaluations: step i reads states_host[i] at T[i] (a scalar T applies to every step) and writes
        outs_host[i].  A tensor may repeat in either list."""
        n = len(states_host)
        if len(outs_host) != n:
            raise ValueError("states_host and outs_host differ in length")
        for t in list(states_host) + list(outs_host):
            if t.device.type != "cpu" or not t.is_contiguous() or t.dtype != torch.complex128 \
                    or tuple(t.shape) != self.state_shape():
                raise ValueError(f"rhs_host_batch needs C-contiguous complex128 host tensors of shape {self.state_shape()}")
        Ts = [float(T)] * n if np.ndim(T) == 0 else [float(x) for x in T]
        if len(Ts) != n:
            raise ValueError("T has the wrong length")
        t_arr = (C.c_double * max(n, 1))(*Ts)
        s_arr = (C.c_void_p * max(n, 1))(*[t.data_ptr() for t in states_host])
        o_arr = (C.c_void_p * max(n, 1))(*[t.data_ptr() for t in outs_host])
        flag = SYMMETRIC_STATE if symmetric else 0
        self._check(self._L.tufrg_rhs_host_batch(self._h, n, t_arr, s_arr, int(mask) | flag, o_arr))
        return outs_host

    # ------------------------------------------------------------------ irrep form factors (C4v)
    IRREPS = ("A1", "A2", "B1", "B2", "E")

    def form_factors(self):
        """(W [n_ff][n_ff], labels [n_ff][3] = (shell, irrep index, partner)): the form factors of the irreducible
        representations of C4v over the bonds; raises (TUFRG_ENOTSUP) for a bond set not closed under the group."""
        n = self.spec.n_ff
        W = np.zeros((n, n))
        lab = np.zeros((n, 3), np.int32)
        self._check(self._L.tufrg_form_factors(self._h, W.ctypes.data, lab.ctypes.data))
        return W, lab

    def irrep_basis(self, state, inverse: bool = False, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """The state with its form factors changed to the irrep combinations, (W x 1) X (W x 1)^T (inverse: back)."""
        st = self._dev(state)
        out = torch.empty_like(st) if out is None else out
        self._check(self._L.tufrg_irrep_basis(self._h, _ptr(st), 1 if inverse else 0, _ptr(out)))
        return out

    # ------------------------------------------------------------------ right-hand side over shards of momenta
    def shard_classes(self) -> np.ndarray:
        """Bond classes R'' (mod Lq) of the shard transforms, [ncls][2]."""
        n = C.c_int()
        self._check(self._L.tufrg_shard_classes(self._h, C.byref(n), None))
        cls = np.zeros((n.value, 2), np.int32)
        self._check(self._L.tufrg_shard_classes(self._h, C.byref(n), cls.ctypes.data))
        return cls

    def shard_transform(self, state_local, q_list, mask: int = CH_P | CH_C) -> torch.Tensor:
        """This shard's part of the Fourier transform to the bond classes, [2][ncls][M][M] complex128 on the device;
        state_local [2][len(q_list)][M][M] holds the rows of the listed momenta."""
        ql = np.ascontiguousarray(q_list, np.int32)
        st = self._dev(state_local)
        if tuple(st.shape) != (2, ql.shape[0], self.M, self.M):
            raise ValueError("state_local must be [2][len(q_list)][M][M]")
        ncls = self.shard_classes().shape[0]
        out = torch.zeros((2, ncls, self.M, self.M), dtype=torch.complex128, device=st.device)
        self._check(self._L.tufrg_rhs_shard_transform(self._h, _ptr(st), ql.shape[0], ql.ctypes.data, int(mask), _ptr(out)))
        return out

    def shard_finish(self, T: float, state_local, q_list, xr, mask: int = CH_P | CH_C) -> torch.Tensor:
        """dX/dT of the listed momenta, [2][len(q_list)][M][M], from their rows and the transforms summed over all
        shards."""
        ql = np.ascontiguousarray(q_list, np.int32)
        st = self._dev(state_local)
        xr = self._dev(xr)
        out = torch.empty_like(st)
        self._check(self._L.tufrg_rhs_shard_finish(self._h, float(T), _ptr(st), ql.shape[0], ql.ctypes.data, _ptr(xr),
                                                   int(mask), _ptr(out)))
        return out

    PHASES = ("fermi", "loops", "loop_reduce", "dft", "project", "vlv", "rk", "sym_scatter")

    def timing_begin(self):
        self._check(self._L.tufrg_timing_begin(self._h))

    def timing_end(self):
        ms = np.zeros(len(self.PHASES))
        nl, nloop = C.c_longlong(), C.c_longlong()
        self._check(self._L.tufrg_timing_end(self._h, ms.ctypes.data, len(ms), C.byref(nl), C.byref(nloop)))
        return dict(zip(self.PHASES, ms.tolist())), nl.value, nloop.value

    def flow(self, T0: float = FLOW_T0, T_end: float = FLOW_T_END, rtol: float = FLOW_RTOL, atol: float = FLOW_ATOL,
             h0: float = -0.05, stop: float = FLOW_STOP, mask: int = CH_P | CH_C, max_steps: int = 100000,
             want_state: bool = True, metrics_path: Optional[str] = None, checkpoint_path: Optional[str] = None,
             checkpoint_every: int = 0, resume_from: Optional[str] = None, stop_after: int = 0):
        """The adaptive flow (tufrg_flow).  With metrics_path, checkpoint_path or resume_from it runs step by step
        (tufrg_flow_start / tufrg_flow_resume, tufrg_flow_step, tufrg_flow_end): one JSON line per accepted step
        to metrics_path (T, h, err, max|A| per channel, counts), the checkpoint written to checkpoint_path every
        checkpoint_every accepted steps (replacing the previous one), the flow continued from the checkpoint file
        resume_from.  stop_after > 0 ends the run after that many accepted steps of this call (the result is then
        that of an unfinished flow; resume from its checkpoint to continue)."""
        o = FlowOpts(T0, T_end, rtol, atol, h0, stop, int(mask), int(max_steps))
        r = FlowResult()
        st_out = self.zeros_state() if want_state else None
        if not (metrics_path or checkpoint_path or resume_from):
            self._check(self._L.tufrg_flow(self._h, C.byref(o), _ptr(st_out) if want_state else None, C.byref(r)))
            return st_out, {f: getattr(r, f) for f, _ in FlowResult._fields_}
        import json
        import os
        nbytes = self._L.tufrg_flow_checkpoint_bytes(self._h)
        buf = np.empty(nbytes, np.uint8)
        if resume_from:
            data = np.fromfile(resume_from, np.uint8)
            self._check(self._L.tufrg_flow_resume(self._h, C.byref(o), data.ctypes.data, data.size))
        else:
            self._check(self._L.tufrg_flow_start(self._h, C.byref(o)))
        info, amax2 = FlowStepInfo(), np.zeros(2)
        metrics = open(metrics_path, "a") if metrics_path else None
        try:
            done = 0
            while True:
                self._check(self._L.tufrg_flow_step(self._h, C.byref(info)))
                if info.accepted:
                    done += 1
                    if metrics:
                        self._check(self._L.tufrg_flow_amax_channels(self._h, amax2.ctypes.data))
                        metrics.write(json.dumps({"step": info.n_steps, "T": info.T, "h": info.h, "err": info.err,
                                                  "amax": info.amax, "amax_P": float(amax2[0]),
                                                  "amax_C": float(amax2[1]), "n_reject": info.n_reject,
                                                  "status": info.status}) + "\n")
                    if checkpoint_path and checkpoint_every > 0 and info.n_steps % checkpoint_every == 0:
                        self._check(self._L.tufrg_flow_save(self._h, buf.ctypes.data, nbytes))
                        tmp = checkpoint_path + ".tmp"
                        buf.tofile(tmp)
                        os.replace(tmp, checkpoint_path)
                if info.status != 0 or (stop_after > 0 and done >= stop_after):
                    break
        finally:
            if metrics:
                metrics.close()
            st = self._L.tufrg_flow_end(self._h, _ptr(st_out) if want_state else None, C.byref(r))
        self._check(st)
        return st_out, {f: getattr(r, f) for f, _ in FlowResult._fields_}


def flow_batch(models, T0: float = FLOW_T0, T_end: float = FLOW_T_END, rtol: float = FLOW_RTOL,
               atol: float = FLOW_ATOL, h0: float = -0.05, stop: float = FLOW_STOP, mask: int = CH_P | CH_C,
               max_steps: int = 100000):
    """Run the adaptive flows of several models together (tufrg_flow_batch).

    Each model should have been created on its own torch stream so that the flows overlap.
    Returns one result dict per model."""
    if not models:
        return []
    L = models[0]._L
    arr = (C.c_void_p * len(models))(*[m._h.value for m in models])
    res = (FlowResult * len(models))()
    o = FlowOpts(T0, T_end, rtol, atol, h0, stop, int(mask), int(max_steps))
    st = L.tufrg_flow_batch(arr, len(models), C.byref(o), res)
    if st != 0:
        msgs = "; ".join(m._L.tufrg_last_error(m._h).decode() for m in models if m._L.tufrg_last_error(m._h))
        raise TufrgError(st, msgs)
    return [{f: getattr(r, f) for f, _ in FlowResult._fields_} for r in res]
