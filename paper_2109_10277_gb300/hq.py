"""Python binding of libhq (include/hq.h): argument marshalling only.

Every step of the quasi-static slice loop runs in the CUDA kernels of libhq.so;
PyTorch provides device memory (tensors) and the stream.  There is no fallback:
if the library is missing or the device is not sm_103a the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhq.so")

HQ_PREC_FP64 = 0
HQ_PREC_FP32_BF16X3 = 1
HQ_PREC_FP32_TF32X3 = 2
# precision names of Grid: "fp64", "fp32" (= "bf16x3", the FP32 path with bf16x3 tensor-core DST
# operands) and "tf32x3" (the same FP32 path with TF32x3 operands)
PRECISIONS = {"fp64": HQ_PREC_FP64, "fp32": HQ_PREC_FP32_BF16X3, "bf16x3": HQ_PREC_FP32_BF16X3,
              "tf32x3": HQ_PREC_FP32_TF32X3}
STATUS = {0: "HQ_OK", 1: "HQ_ERR_ARG", 2: "HQ_ERR_CUDA", 3: "HQ_ERR_OOM", 4: "HQ_ERR_NUMERIC",
          5: "HQ_ERR_TIMEOUT", 6: "HQ_ERR_STATE", 7: "HQ_ERR_UNSUPPORTED"}
FIELDS = ("rho", "jx", "jy", "jz", "chi", "psi", "exmby", "eypbx", "ez", "bx", "by", "bz")
EXPORTS = ("hq_grid_create", "hq_grid_destroy", "hq_advance_slice", "hq_beam_deposit", "hq_solve_fields",
           "hq_store_fields", "hq_push_beams", "hq_witness_accumulate", "hq_sweep_step", "hq_poisson_solve",
           "hq_plasma_state", "hq_profile_enable", "hq_profile_read", "hq_sync", "hq_last_error",
           "hq_poisson_solve_static", "hq_sweep_forward_ckpt", "hq_sweep_adjoint", "hq_beam_moments",
           "hq_beam_slices", "hq_sweep_slices", "hq_pc_residuals")
KERNEL_CLASSES = ("final", "trial", "dst", "field", "beam", "other")


class SpeciesDesc(C.Structure):
    _fields_ = [("charge", C.c_double), ("mass", C.c_double), ("n0_scale", C.c_double),
                ("ppc_x", C.c_int32), ("ppc_y", C.c_int32), ("radial_profile", C.POINTER(C.c_double)),
                ("n_profile", C.c_int32), ("profile_rmax", C.c_double), ("neutralize", C.c_int32)]


class GridDesc(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nzeta", C.c_int32),
                ("xmin", C.c_double), ("xmax", C.c_double), ("ymin", C.c_double), ("ymax", C.c_double),
                ("zeta_min", C.c_double), ("zeta_max", C.c_double),
                ("shape_order", C.c_int32), ("ppc_x", C.c_int32), ("ppc_y", C.c_int32),
                ("radial_profile", C.POINTER(C.c_double)), ("n_profile", C.c_int32), ("profile_rmax", C.c_double),
                ("n0_scale", C.c_double), ("n_pc_iter", C.c_int32), ("pc_mix", C.c_double),
                ("psi_guard", C.c_double), ("precision", C.c_int32), ("bperp_solver", C.c_int32),
                ("resort_every", C.c_int32), ("deterministic", C.c_int32),
                ("species", C.POINTER(SpeciesDesc)), ("n_species", C.c_int32), ("pc_residuals", C.c_int32)]


class BeamView(C.Structure):
    _fields_ = [("n", C.c_int64)] + [(k, C.c_void_p) for k in ("x", "y", "zeta", "ux", "uy", "uz", "w")] + \
               [("charge", C.c_double), ("mass", C.c_double)]


class FieldOut(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in FIELDS]


class Profile(C.Structure):
    _fields_ = [("ms", C.c_double * 8), ("launches", C.c_int64 * 8)]


class PlasmaView(C.Structure):
    _fields_ = [("n", C.c_int64), ("x", C.c_void_p), ("y", C.c_void_p), ("psi", C.c_void_p),
                ("ux", C.c_void_p), ("uy", C.c_void_p), ("w", C.c_void_p), ("alive", C.c_void_p),
                ("origin", C.c_void_p)]


_lib = None


def load() -> C.CDLL:
    """Load libhq.so (built in-tree by paper_2109_10277_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2109_10277_gb300.build`")
        lib = C.CDLL(LIB_PATH)
        P, I32, I64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_double
        sig = {
            "hq_grid_create": (C.POINTER(GridDesc), P, C.POINTER(P)),
            "hq_grid_destroy": (P,),
            "hq_advance_slice": (P, I32),
            "hq_beam_deposit": (P, C.POINTER(BeamView), I32, I32),
            "hq_solve_fields": (P, I32),
            "hq_store_fields": (P, C.POINTER(FieldOut), I64),
            "hq_push_beams": (P, C.POINTER(BeamView), I32, I32, D),
            "hq_witness_accumulate": (P, C.POINTER(BeamView), I32, P),
            "hq_sweep_step": (P, C.POINTER(BeamView), I32, D, C.POINTER(FieldOut), I32, P),
            "hq_poisson_solve": (P, P, P, I32),
            "hq_plasma_state": (P, C.POINTER(PlasmaView)),
            "hq_profile_enable": (P, I32),
            "hq_profile_read": (P, C.POINTER(Profile)),
            "hq_sync": (P, C.POINTER(I64)),
            "hq_poisson_solve_static": (P, P, I32, I32, D, D, I32, P),
            "hq_sweep_forward_ckpt": (P, C.POINTER(BeamView), I32, I32, P, I32),
            "hq_sweep_adjoint": (P, C.POINTER(BeamView), I32, I32, C.POINTER(D), C.POINTER(FieldOut), C.POINTER(P), P, P,
                                 P),
            "hq_beam_moments": (P, C.POINTER(BeamView), P),
            "hq_beam_slices": (P, C.POINTER(BeamView), P),
            "hq_pc_residuals": (P, C.POINTER(C.c_double), C.c_int32),
            "hq_sweep_slices": (P, C.POINTER(BeamView), C.c_int32, C.POINTER(BeamView), C.c_int32, C.c_int32,
                                C.c_int32, C.c_double, C.POINTER(FieldOut), C.c_int32, P),
        }
        for name, args in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = list(args)
            fn.restype = C.c_int
        lib.hq_last_error.argtypes = [P]
        lib.hq_last_error.restype = C.c_char_p
        _lib = lib
    return _lib


class HQError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _check(st: int, handle) -> None:
    if st != 0:
        msg = load().hq_last_error(handle)
        raise HQError(st, msg.decode() if msg else "")


def _ptr(t: Optional[torch.Tensor]) -> Optional[int]:
    return None if t is None else t.data_ptr()


class _CudaArray:
    """Zero-copy view of library-owned device memory (for hq_plasma_state)."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False), "version": 3}


class Beam:
    """One beam species: float64 CUDA tensors x, y, zeta, ux, uy, uz, w (updated in place by pushes)."""

    def __init__(self, arrays: dict, device: str = "cuda", charge: Optional[float] = None,
                 mass: Optional[float] = None):
        self.t = {k: torch.as_tensor(arrays[k], dtype=torch.float64, device=device).contiguous()
                  for k in ("x", "y", "zeta", "ux", "uy", "uz", "w")}
        self.charge = float(arrays.get("charge", -1.0) if charge is None else charge)
        self.mass = float(arrays.get("mass", 1.0) if mass is None else mass)

    @property
    def n(self) -> int:
        return int(self.t["x"].numel())

    def view(self) -> BeamView:
        return BeamView(self.n, *[self.t[k].data_ptr() for k in ("x", "y", "zeta", "ux", "uy", "uz", "w")],
                        self.charge, self.mass)


def _beam_array(beams: Sequence[Beam]):
    arr = (BeamView * max(1, len(beams)))()
    for i, b in enumerate(beams):
        arr[i] = b.view()
    return arr


class Grid:
    """A quasi-static grid (plasma slice, field slices, DST scratch) on the current CUDA device."""

    def __init__(self, params: dict, precision: str = "fp64", stream: Optional[torch.cuda.Stream] = None):
        lib = load()
        if precision not in PRECISIONS:
            raise ValueError(f"precision must be one of {sorted(PRECISIONS)}")
        self.precision = precision
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        prof = params.get("radial_profile")
        self._prof = (C.c_double * len(prof))(*prof) if prof is not None else None
        # plasma species: dicts with charge, mass, n0_scale, ppc_x, ppc_y, radial_profile,
        # profile_rmax, neutralize (the library copies them)
        sps = list(params.get("species") or [])
        self._sp_prof = []
        self._sp = (SpeciesDesc * max(1, len(sps)))()
        for k, sp in enumerate(sps):
            pr = sp.get("radial_profile")
            arr = (C.c_double * len(pr))(*pr) if pr is not None else None
            self._sp_prof.append(arr)
            self._sp[k] = SpeciesDesc(float(sp.get("charge", -1.0)), float(sp.get("mass", 1.0)),
                                      float(sp.get("n0_scale", 1.0)), int(sp.get("ppc_x", 1)), int(sp.get("ppc_y", 1)),
                                      C.cast(arr, C.POINTER(C.c_double)) if arr is not None else None,
                                      len(pr) if pr is not None else 0, float(sp.get("profile_rmax", 0.0)),
                                      int(bool(sp.get("neutralize", True))))
        d = GridDesc(
            int(params["nx"]), int(params["ny"]), int(params["nzeta"]),
            float(params["xmin"]), float(params["xmax"]), float(params["ymin"]), float(params["ymax"]),
            float(params["zeta_min"]), float(params["zeta_max"]),
            int(params.get("shape_order", 1)), int(params.get("ppc_x", 1)), int(params.get("ppc_y", 1)),
            C.cast(self._prof, C.POINTER(C.c_double)) if self._prof is not None else None,
            len(prof) if prof is not None else 0, float(params.get("profile_rmax", 0.0)),
            float(params.get("n0_scale", 1.0)), int(params.get("n_pc_iter", 5)), float(params.get("pc_mix", 0.05)),
            float(params.get("psi_guard", 0.02)),
            PRECISIONS[precision],
            {"pc": 0, "explicit": 1}[params.get("bperp_solver", "pc")], int(params.get("resort_every", 0)),
            int(params.get("deterministic", 0)),
            C.cast(self._sp, C.POINTER(SpeciesDesc)) if sps else None, len(sps), int(params.get("pc_residuals", 0)))
        self.params = dict(params)
        self.nx, self.ny, self.nzeta = d.nx, d.ny, d.nzeta
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        _check(lib.hq_grid_create(C.byref(d), C.c_void_p(self.stream.cuda_stream), C.byref(h)), None)
        self.h = h

    def close(self) -> None:
        if getattr(self, "h", None):
            load().hq_grid_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _out(self, out: Optional[dict]):
        if out is None:
            return None
        fo = FieldOut()
        for k in FIELDS:
            t = out.get(k)
            if t is not None:
                assert t.dtype == self.dtype and t.is_cuda and t.is_contiguous()
                setattr(fo, k, t.data_ptr())
        return fo

    def alloc_out(self, names: Sequence[str] = FIELDS, nslots: Optional[int] = None) -> dict:
        n = self.nzeta if nslots is None else nslots
        return {k: torch.zeros((n, self.ny, self.nx), dtype=self.dtype, device="cuda") for k in names}

    # fine-grained steps (Sec. 2 enumerate)
    def advance(self, slice_: int) -> None:
        _check(load().hq_advance_slice(self.h, slice_), self.h)

    def beam_deposit(self, beams: Sequence[Beam], slice_: int) -> None:
        self._beams = _beam_array(beams)
        _check(load().hq_beam_deposit(self.h, self._beams, len(beams), slice_), self.h)

    def solve(self, slice_: int) -> None:
        _check(load().hq_solve_fields(self.h, slice_), self.h)

    def store(self, out: dict, slot: int) -> None:
        fo = self._out(out)
        _check(load().hq_store_fields(self.h, C.byref(fo), slot), self.h)

    def push_beams(self, beams: Sequence[Beam], slice_: int, dt: float) -> None:
        arr = _beam_array(beams)
        _check(load().hq_push_beams(self.h, arr, len(beams), slice_, float(dt)), self.h)

    def witness_accumulate(self, beam: Beam, slice_: int, sums: torch.Tensor) -> None:
        v = beam.view()
        _check(load().hq_witness_accumulate(self.h, C.byref(v), slice_, C.c_void_p(sums.data_ptr())), self.h)

    def sweep(self, beams: Sequence[Beam] = (), dt: float = 0.0, out: Optional[dict] = None,
              witness: int = -1, witness_sums: Optional[torch.Tensor] = None) -> None:
        arr = _beam_array(beams)
        fo = self._out(out)
        _check(load().hq_sweep_step(self.h, arr, len(beams), float(dt), C.byref(fo) if fo is not None else None,
                                    int(witness), C.c_void_p(_ptr(witness_sums)) if witness_sums is not None else None),
               self.h)

    def sweep_slices(self, beams: Sequence[Beam], begin: int, end: int, next_beams: Sequence[Beam] = (),
                     dt: float = 0.0, out: Optional[dict] = None, witness: int = -1,
                     witness_sums: Optional[torch.Tensor] = None) -> None:
        """Slices [begin, end) of a sweep (hq_sweep_slices): one box of the temporal pipeline."""
        arr = _beam_array(beams)
        nxt = _beam_array(next_beams)
        fo = self._out(out)
        _check(load().hq_sweep_slices(self.h, arr, len(beams), nxt, len(next_beams), int(begin), int(end), float(dt),
                                      C.byref(fo) if fo is not None else None, int(witness),
                                      C.c_void_p(_ptr(witness_sums)) if witness_sums is not None else None), self.h)

    def forward_ckpt(self, beams: Sequence[Beam], witness: int, sums: torch.Tensor, ckpt_every: int) -> None:
        """Checkpointed forward sweep (no field output); sums (device float64[3]) += witness sums."""
        arr = _beam_array(beams)
        _check(load().hq_sweep_forward_ckpt(self.h, arr, len(beams), int(witness), C.c_void_p(sums.data_ptr()),
                                            int(ckpt_every)), self.h)
        self._adj_beams = arr

    def adjoint(self, beams: Sequence[Beam], witness: int, dl_dsums: Optional[Sequence[float]], plasma: bool = True,
                dl_dfields: Optional[dict] = None) -> dict:
        """Reverse sweep of the last forward_ckpt: gradients w.r.t. beam and plasma weights,
        the density scale n0 and the radial profile, of a loss with dL/d(witness sums) dl_dsums
        and, optionally, dL/d(field) seeds dl_dfields (name -> (nzeta, ny, nx) field-type tensor)."""
        arr = _beam_array(beams)
        wb = [torch.zeros(b.n, dtype=torch.float64, device="cuda") for b in beams]
        ptrs = (C.c_void_p * max(1, len(beams)))(*[t.data_ptr() for t in wb])
        np_ = self.nx * self.ny * int(self.params.get("ppc_x", 1)) * int(self.params.get("ppc_y", 1))
        wp = torch.zeros(np_, dtype=torch.float64, device="cuda") if plasma else None
        dn0 = torch.zeros(1, dtype=torch.float64, device="cuda")
        prof = self.params.get("radial_profile")
        dprof = torch.zeros(len(prof), dtype=torch.float64, device="cuda") if prof is not None else None
        sb = (C.c_double * 3)(*[float(v) for v in dl_dsums]) if dl_dsums is not None else None
        fo = self._out(dl_dfields)
        _check(load().hq_sweep_adjoint(self.h, arr, len(beams), int(witness), sb,
                                       C.byref(fo) if fo is not None else None, ptrs,
                                       C.c_void_p(wp.data_ptr()) if wp is not None else None,
                                       C.c_void_p(dn0.data_ptr()),
                                       C.c_void_p(dprof.data_ptr()) if dprof is not None else None), self.h)
        return {"beam_w": wb, "plasma_w": wp, "n0_scale": dn0, "profile": dprof}

    def pc_residuals(self) -> list:
        """Per slice of the last sweep: ||B_m - B_m-1|| / ||B_m|| of the last predictor-corrector iteration."""
        out = (C.c_double * self.nzeta)()
        _check(load().hq_pc_residuals(self.h, out, self.nzeta), self.h)
        return list(out)

    def beam_slices(self, beam: Beam) -> torch.Tensor:
        """Slice of every particle (int32 CUDA tensor): 0..nzeta-1 inside, -1 ahead, nzeta behind, -2 not finite."""
        out = torch.empty(beam.n, dtype=torch.int32, device="cuda")
        v = beam.view()
        _check(load().hq_beam_slices(self.h, C.byref(v), C.c_void_p(out.data_ptr()) if beam.n else None), self.h)
        return out

    def beam_moments(self, beam: Beam) -> torch.Tensor:
        """Weighted raw moments of a beam (device float64[11], see hq_beam_moments)."""
        m = torch.zeros(11, dtype=torch.float64, device="cuda")
        v = beam.view()
        _check(load().hq_beam_moments(self.h, C.byref(v), C.c_void_p(m.data_ptr())), self.h)
        return m

    def poisson_solve(self, src: torch.Tensor) -> torch.Tensor:
        assert src.dtype == self.dtype and src.is_cuda and src.is_contiguous() and src.dim() == 3
        dst = torch.empty_like(src)
        _check(load().hq_poisson_solve(self.h, C.c_void_p(src.data_ptr()), C.c_void_p(dst.data_ptr()),
                                       src.shape[0]), self.h)
        return dst

    def plasma_state(self, initial_order: bool = True) -> dict:
        """Copies of the plasma slice arrays (synchronizes the grid's stream).  A grid that
        re-sorts its plasma also returns "origin" (each entry's index in the initial placement)
        and, with initial_order, the arrays put back in that placement's order."""
        v = PlasmaView()
        _check(load().hq_plasma_state(self.h, C.byref(v)), self.h)
        self.sync()
        ft = "<f8" if self.precision == "fp64" else "<f4"
        n = int(v.n)
        out = {}
        for k, ts in (("x", "<f8"), ("y", "<f8"), ("psi", "<f8"), ("ux", ft), ("uy", ft), ("w", ft), ("alive", "|u1")):
            out[k] = torch.as_tensor(_CudaArray(getattr(v, k), n, ts), device="cuda").clone()
        if v.origin:
            org = torch.as_tensor(_CudaArray(v.origin, n, "<i4"), device="cuda").clone().to(torch.int64)
            if initial_order:
                for k in list(out):
                    t = torch.empty_like(out[k])
                    t[org] = out[k]
                    out[k] = t
            out["origin"] = org
        return out

    def profile(self, on: bool) -> None:
        """Start (on=True) or stop per-kernel-class CUDA-event timing; resets the counters."""
        _check(load().hq_profile_enable(self.h, 1 if on else 0), self.h)

    def profile_read(self) -> dict:
        """{class: (ms, launches)} accumulated since the last profile() call."""
        pr = Profile()
        _check(load().hq_profile_read(self.h, C.byref(pr)), self.h)
        return {k: (float(pr.ms[i]), int(pr.launches[i])) for i, k in enumerate(KERNEL_CLASSES)}

    def sync(self) -> int:
        rm = C.c_int64()
        _check(load().hq_sync(self.h, C.byref(rm)), self.h)
        return int(rm.value)


def emittance(moments) -> tuple:
    """Normalised rms emittances (eps_x, eps_y) from hq_beam_moments' eleven sums (host
    arithmetic on scalars): eps^2 = <dx^2><du^2> - <dx du>^2, centred and weight-averaged."""
    m = [float(v) for v in moments]
    out = []
    for a, b, aa, bb, ab in ((1, 3, 5, 7, 9), (2, 4, 6, 8, 10)):
        ma, mb = m[a] / m[0], m[b] / m[0]
        vaa, vbb, vab = m[aa] / m[0] - ma * ma, m[bb] / m[0] - mb * mb, m[ab] / m[0] - ma * mb
        out.append(max(vaa * vbb - vab * vab, 0.0) ** 0.5)
    return tuple(out)


def witness_loss_grad(kind: str, s0: float, s1: float, s2: float):
    """Loss from the witness sums and dL/d(S0, S1, S2): "mean" = S1/S0, "mean+rms" adds
    sqrt(S2/S0 - (S1/S0)^2) (host arithmetic on three scalars)."""
    mean = s1 / s0
    if kind == "mean":
        return mean, (-s1 / (s0 * s0), 1.0 / s0, 0.0)
    var = max(s2 / s0 - mean * mean, 0.0)
    sd = var ** 0.5
    if sd == 0.0:
        return mean, (-s1 / (s0 * s0), 1.0 / s0, 0.0)
    dvar = (-s2 / (s0 * s0) + 2.0 * mean * s1 / (s0 * s0), -2.0 * mean / s0, 1.0 / s0)
    return mean + sd, (-s1 / (s0 * s0) + dvar[0] / (2 * sd), 1.0 / s0 + dvar[1] / (2 * sd), dvar[2] / (2 * sd))


class SweepLoss(torch.autograd.Function):
    """Witness loss of one quasi-static sweep, differentiable w.r.t. the beam weights and the
    plasma density scale / radial profile through the hand-written reverse-zeta adjoint.

    apply(grid, beams, witness, kind, ckpt_every, n0_scale, profile, *beam_weights) -> loss.
    n0_scale (0-d) and profile (1-d or an empty tensor) must hold the values the grid was
    created with; beam_weights[i] are copied into beams[i] before the sweep."""

    @staticmethod
    def forward(ctx, grid, beams, witness, kind, ckpt_every, n0_scale, profile, *weights):
        for b, w in zip(beams, weights):
            b.t["w"].copy_(w.detach())
        sums = torch.zeros(3, dtype=torch.float64, device="cuda")
        grid.forward_ckpt(beams, witness, sums, ckpt_every)
        s = [float(v) for v in sums.cpu()]
        loss, dls = witness_loss_grad(kind, *s)
        ctx.grid, ctx.beams, ctx.witness, ctx.dls = grid, beams, witness, dls
        ctx.has_prof = profile.numel() > 0
        ctx.n0_like = (n0_scale.shape, n0_scale.device, n0_scale.dtype)
        ctx.prof_like = (profile.device, profile.dtype)
        return torch.tensor(loss, dtype=torch.float64, device=weights[0].device if weights else "cuda")

    @staticmethod
    def backward(ctx, gl):
        g = float(gl)
        res = ctx.grid.adjoint(ctx.beams, ctx.witness, [g * v for v in ctx.dls], plasma=True)
        shape, dev, dt = ctx.n0_like
        dn0 = res["n0_scale"][0].to(device=dev, dtype=dt).reshape(shape)
        dprof = res["profile"].to(device=ctx.prof_like[0], dtype=ctx.prof_like[1]) if ctx.has_prof else None
        return (None, None, None, None, None, dn0, dprof, *res["beam_w"])
