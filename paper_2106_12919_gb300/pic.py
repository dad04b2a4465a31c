"""Thin ctypes binding of libpic (include/pic.h): argument marshalling only.

Every entry point of the C ABI has a same-named method on :class:`Context`
(``pic_step`` -> ``Context.step`` ...).  Field and particle arguments are
torch CUDA tensors (contiguous; float64 for the pic_step family, float32 and int32 cells for
the pic_step32 family); the binding passes their device pointers and the context's stream.  All computation happens in the CUDA
library: if it cannot be loaded this module raises at import time.
"""
import ctypes
import os

import torch

from . import build as _build

PIC_OK = 0
PIC_FP64, PIC_FP32 = 0, 1
PIC_PUSHER_BORIS, PIC_PUSHER_VAY = 0, 1
PIC_CYCLE_HYBRID, PIC_CYCLE_NODAL, PIC_CYCLE_STAGGERED, PIC_CYCLE_HYBRID_FDTD = 0, 1, 2, 3
STATUS = {0: "PIC_OK", -1: "PIC_ERR_ARG", -2: "PIC_ERR_UNSUPPORTED", -3: "PIC_ERR_NOMEM",
          -4: "PIC_ERR_CUDA", -5: "PIC_ERR_CAPACITY", -6: "PIC_ERR_TIMEOUT", -7: "PIC_ERR_NONFINITE"}
STANDARD, GALILEAN, AVERAGED = 0, 1, 2

_d3 = ctypes.c_double * 3
_i3 = ctypes.c_int32 * 3
_l3 = ctypes.c_int64 * 3
_vp = ctypes.c_void_p


class PicExt(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("spectral_order", _i3), ("precision", ctypes.c_int32),
                ("c", ctypes.c_double), ("eps0", ctypes.c_double), ("tile", _i3),
                ("sort_interval", ctypes.c_int32), ("cuda_stream", _vp), ("filter_passes", ctypes.c_int32),
                ("pusher", ctypes.c_int32), ("cycle", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class PicSpecies(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("q", ctypes.c_double), ("m", ctypes.c_double),
                ("x", _vp), ("y", _vp), ("z", _vp), ("ux", _vp), ("uy", _vp), ("uz", _vp), ("w", _vp),
                ("id", _vp)]


class PicSpecies32(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("q", ctypes.c_double), ("m", ctypes.c_double),
                ("cell", _vp), ("fx", _vp), ("fy", _vp), ("fz", _vp), ("ux", _vp), ("uy", _vp), ("uz", _vp),
                ("w", _vp), ("id", _vp)]


class PicSpeciesAdjoint(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("x", _vp), ("y", _vp), ("z", _vp), ("ux", _vp), ("uy", _vp), ("uz", _vp)]


class PicError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


def _load():
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError("libpic is not built (%s missing): run __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    sig = {
        "pic_ext_default": (None, [P(PicExt)]),
        "pic_init": (ctypes.c_int, [P(_vp), P(ctypes.c_int64), P(ctypes.c_double), ctypes.c_double, ctypes.c_int,
                                    P(ctypes.c_int32), ctypes.c_int, P(ctypes.c_double), P(PicExt)]),
        "pic_destroy": (None, [_vp]),
        "pic_last_error": (ctypes.c_char_p, [_vp]),
        "pic_sync": (ctypes.c_int, [_vp]),
        "pic_step": (ctypes.c_int, [_vp, P(_vp), P(_vp), P(_vp), _vp, P(PicSpecies), ctypes.c_int, ctypes.c_int]),
        "pic_deposit_rho": (ctypes.c_int, [_vp, P(PicSpecies), ctypes.c_int, _vp]),
        "pic_push_deposit": (ctypes.c_int, [_vp, P(_vp), P(_vp), P(PicSpecies), ctypes.c_int, P(_vp), _vp]),
        "pic_bin": (ctypes.c_int, [_vp, P(PicSpecies), _vp]),
        "pic_num_tiles": (ctypes.c_int64, [_vp]),
        "pic_center_to_nodal": (ctypes.c_int, [_vp, P(_vp), P(_vp)]),
        "pic_center_to_yee": (ctypes.c_int, [_vp, P(_vp), P(_vp)]),
        "pic_fft_forward": (ctypes.c_int, [_vp, P(_vp), P(_vp), ctypes.c_int]),
        "pic_fft_inverse": (ctypes.c_int, [_vp, P(_vp), P(_vp), ctypes.c_int]),
        "pic_maxwell_step": (ctypes.c_int, [_vp, P(_vp), P(_vp), P(_vp), _vp, _vp, P(_vp), P(_vp)]),
        "pic_coefficient": (ctypes.c_int, [_vp, ctypes.c_char_p, _vp]),
        "pic_field_energy": (ctypes.c_int, [_vp, P(_vp), P(_vp), P(ctypes.c_int64), P(ctypes.c_int64),
                                            P(ctypes.c_double)]),
        "pic_total_charge": (ctypes.c_int, [_vp, _vp, P(ctypes.c_double)]),
        "pic_timing": (ctypes.c_int, [_vp, ctypes.c_int]),
        "pic_center_to_nodal_static": (ctypes.c_int, [P(ctypes.c_int64), P(ctypes.c_int32), P(_vp), P(_vp), _vp]),
        "pic_step32": (ctypes.c_int, [_vp, P(_vp), P(_vp), P(_vp), _vp, P(PicSpecies32), ctypes.c_int, ctypes.c_int]),
        "pic_deposit_rho32": (ctypes.c_int, [_vp, P(PicSpecies32), ctypes.c_int, _vp]),
        "pic_push_deposit32": (ctypes.c_int, [_vp, P(_vp), P(_vp), P(PicSpecies32), ctypes.c_int, P(_vp), _vp]),
        "pic_bin32": (ctypes.c_int, [_vp, P(PicSpecies32), _vp]),
        "pic_fft_forward32": (ctypes.c_int, [_vp, P(_vp), P(_vp), ctypes.c_int]),
        "pic_fft_inverse32": (ctypes.c_int, [_vp, P(_vp), P(_vp), ctypes.c_int]),
        "pic_field_energy32": (ctypes.c_int, [_vp, P(_vp), P(_vp), P(ctypes.c_int64), P(ctypes.c_int64),
                                              P(ctypes.c_double)]),
        "pic_total_charge32": (ctypes.c_int, [_vp, _vp, P(ctypes.c_double)]),
        "pic_adjoint_step": (ctypes.c_int, [_vp, P(_vp), P(_vp), P(PicSpecies), ctypes.c_int, P(_vp), P(_vp), _vp,
                                            P(PicSpeciesAdjoint)]),
        "pic_timing_read": (ctypes.c_int, [_vp, ctypes.c_char_p, P(ctypes.c_double), P(ctypes.c_int64)]),
        "pic_stencil_extent": (ctypes.c_int, [_vp, ctypes.c_char_p, ctypes.c_int, P(ctypes.c_double)]),
        "pic_axis_tables": (ctypes.c_int, [_vp, ctypes.c_int, P(ctypes.c_double), P(ctypes.c_double),
                                           P(ctypes.c_double)]),
        "pic_vacuum_dispersion": (ctypes.c_int, [_vp, ctypes.c_int, P(ctypes.c_double)]),
        "pic_beam_rms": (ctypes.c_int, [_vp, P(PicSpecies), P(ctypes.c_double)]),
        "pic_beam_rms32": (ctypes.c_int, [_vp, P(PicSpecies32), P(ctypes.c_double)]),
        "pic_species32_from_species": (ctypes.c_int, [_vp, P(PicSpecies), P(PicSpecies32)]),
        "pic_species32_to_species": (ctypes.c_int, [_vp, P(PicSpecies32), P(PicSpecies)]),
        "pic_field_energy_adjoint": (ctypes.c_int, [_vp, P(_vp), P(_vp), P(ctypes.c_int64), P(ctypes.c_int64),
                                                    ctypes.c_double, P(_vp), P(_vp)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


LIB = _load()
EXPORTS = ("pic_ext_default", "pic_init", "pic_destroy", "pic_last_error", "pic_sync", "pic_step",
           "pic_deposit_rho", "pic_push_deposit", "pic_bin", "pic_num_tiles", "pic_center_to_nodal",
           "pic_center_to_yee", "pic_fft_forward", "pic_fft_inverse", "pic_maxwell_step",
           "pic_coefficient", "pic_field_energy", "pic_total_charge", "pic_timing", "pic_timing_read",
           "pic_center_to_nodal_static", "pic_step32", "pic_deposit_rho32", "pic_push_deposit32", "pic_bin32",
           "pic_fft_forward32", "pic_fft_inverse32", "pic_field_energy32", "pic_total_charge32",
           "pic_adjoint_step", "pic_stencil_extent", "pic_axis_tables", "pic_vacuum_dispersion", "pic_beam_rms",
           "pic_beam_rms32", "pic_species32_from_species", "pic_species32_to_species", "pic_field_energy_adjoint")


def _ptr(t, n=None):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_cuda or t.dtype not in (torch.float64, torch.int64, torch.float32, torch.int32) \
            or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA float/int tensor, got %s %s" % (t.device, t.dtype))
    if n is not None and t.numel() != n:
        raise ValueError("expected %d elements, got %d" % (n, t.numel()))
    return t.data_ptr()


def _parr(ts, n=None):
    arr = (_vp * len(ts))()
    for i, t in enumerate(ts):
        arr[i] = _ptr(t, n)
    return arr


def center_to_nodal_static(shape, centering_order, F, out, stream=None):
    """pic_center_to_nodal_static: allocation-free Yee -> nodal centering (no context).

    Returns the pic_status code (0 on success); raises nothing so that callers can
    inspect PIC_ERR_CAPACITY for grids beyond the static scratch.
    """
    n = int(shape[0]) * int(shape[1]) * int(shape[2])
    s = stream if stream is not None else torch.cuda.current_stream()
    return LIB.pic_center_to_nodal_static(_l3(*shape), _i3(*centering_order), _parr(F, n), _parr(out, n),
                                          s.cuda_stream)


class Species:
    """One particle species: torch CUDA float64 tensors x, y, z, ux, uy, uz, w (+ optional int64 id)."""

    def __init__(self, x, y, z, ux, uy, uz, w, q, m, id=None):
        self.x, self.y, self.z, self.ux, self.uy, self.uz, self.w = x, y, z, ux, uy, uz, w
        self.q, self.m, self.id = float(q), float(m), id

    @property
    def n(self):
        return self.x.numel()

    def arrays(self):
        return [self.x, self.y, self.z, self.ux, self.uy, self.uz, self.w]

    def c_struct(self):
        n = self.n
        p = [_ptr(a, n) for a in self.arrays()]
        return PicSpecies(n, self.q, self.m, *p, _ptr(self.id, n) if self.id is not None else None)


class Species32:
    """One FP32-form species: int32 linear cell index, float32 offsets fx, fy, fz in [0, 1),
    float32 ux, uy, uz, w (+ optional int64 id)."""

    def __init__(self, cell, fx, fy, fz, ux, uy, uz, w, q, m, id=None):
        self.cell, self.fx, self.fy, self.fz = cell, fx, fy, fz
        self.ux, self.uy, self.uz, self.w = ux, uy, uz, w
        self.q, self.m, self.id = float(q), float(m), id

    @property
    def n(self):
        return self.cell.numel()

    def arrays(self):
        return [self.cell, self.fx, self.fy, self.fz, self.ux, self.uy, self.uz, self.w]

    def c_struct(self):
        n = self.n
        p = [_ptr(a, n) for a in self.arrays()]
        return PicSpecies32(n, self.q, self.m, *p, _ptr(self.id, n) if self.id is not None else None)

    @staticmethod
    def from_positions(ctx, x, y, z, ux, uy, uz, w, q, m, id=None):
        """FP64 positions, momenta and weights (host arrays or CUDA tensors) -> a new FP32-form
        species on the device, split by pic_species32_from_species on ctx's stream."""
        return ctx.species32_from_species(Species(*[_as_dev64(a) for a in (x, y, z, ux, uy, uz, w)], q, m, id=id))

    def positions(self, ctx):
        """Host FP64 positions [x, y, z] = (cell + offset) dx, formed on the device by
        pic_species32_to_species."""
        s64 = ctx.species32_to_species(self)
        ctx.sync()
        return [s64.x.cpu().numpy(), s64.y.cpu().numpy(), s64.z.cpu().numpy()]


def _as_dev64(a):
    """A host array or tensor as a contiguous CUDA float64 tensor (a copy, no arithmetic)."""
    if isinstance(a, torch.Tensor):
        return a.to(device="cuda", dtype=torch.float64).contiguous()
    import numpy as np
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _species_array(species):
    if species and isinstance(species[0], Species32):
        arr = (PicSpecies32 * max(1, len(species)))()
        for i, s in enumerate(species):
            arr[i] = s.c_struct()
        return arr
    arr = (PicSpecies * max(1, len(species)))()
    for i, s in enumerate(species):
        arr[i] = s.c_struct()
    return arr


class StepGraph:
    """One pic_step / pic_step32 call on fixed arrays, captured into a CUDA graph.

    Every decision of the step is taken on the device (the binning gate included), so the call
    is a fixed sequence of launches on the context's stream and replays exactly; replaying it
    saves the host-side launch cost of each kernel (a step is 20-60 launches).  The call is
    made once uncaptured first (the context allocates its scratch for these particle counts
    then; capture forbids allocation), which advances the arrays by `nsteps`.  replay() runs
    the call again on the current contents of the same arrays, on the current stream.  The
    context must use a stream other than the legacy default stream.
    """

    def __init__(self, ctx, fn, args):
        if ctx.stream.cuda_stream == 0:
            raise ValueError("StepGraph needs a context created on a non-default stream (capture is not "
                             "possible on the legacy default stream)")
        fn(*args)
        ctx.sync()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=ctx.stream):
            fn(*args)
        self.ctx = ctx

    def replay(self):
        self.graph.replay()


class Context:
    """A libpic context (pic_init / pic_destroy) bound to a CUDA stream."""

    def __init__(self, shape, dx, dt, shape_order, centering_order, variant=STANDARD,
                 v_gal=(0.0, 0.0, 0.0), spectral_order=(0, 0, 0), c=1.0, eps0=1.0,
                 tile=(8, 8, 8), sort_interval=20, stream=None, precision=PIC_FP64, filter_passes=0,
                 pusher=0, cycle=0):
        self.shape = tuple(int(n) for n in shape)
        self.dx = tuple(float(d) for d in dx)
        self.ncell = self.shape[0] * self.shape[1] * self.shape[2]
        self.nmode = self.shape[0] * self.shape[1] * (self.shape[2] // 2 + 1)
        self.variant = variant
        self.sort_interval = sort_interval
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        ext = PicExt()
        LIB.pic_ext_default(ctypes.byref(ext))
        ext.spectral_order = _i3(*spectral_order)
        ext.c = c
        ext.eps0 = eps0
        ext.tile = _i3(*tile)
        ext.sort_interval = sort_interval
        ext.precision = precision
        ext.filter_passes = filter_passes
        ext.pusher = pusher
        ext.cycle = cycle
        self.precision = precision
        ext.cuda_stream = self.stream.cuda_stream
        h = _vp()
        st = LIB.pic_init(ctypes.byref(h), _l3(*self.shape), _d3(*dx), dt, shape_order, _i3(*centering_order),
                          variant, _d3(*v_gal), ctypes.byref(ext))
        if st != PIC_OK:
            raise PicError(st, "pic_init failed (see stderr)")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            LIB.pic_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != PIC_OK:
            raise PicError(st, LIB.pic_last_error(self.h).decode())

    def sync(self):
        self._check(LIB.pic_sync(self.h))

    def step(self, E, B, J, rho, species, nsteps):
        """pic_step: E, B, J lists of 3 Yee arrays, rho nodal; species a list of Species."""
        n = self.ncell
        self._check(LIB.pic_step(self.h, _parr(E, n), _parr(B, n), _parr(J, n) if J is not None else None,
                                 _ptr(rho, n),
                                 _species_array(species), len(species), nsteps))

    def deposit_rho(self, species, rho):
        self._check(LIB.pic_deposit_rho(self.h, _species_array(species), len(species), _ptr(rho, self.ncell)))

    def push_deposit(self, En, Bn, species, Jn, rho):
        n = self.ncell
        self._check(LIB.pic_push_deposit(self.h, _parr(En, n), _parr(Bn, n), _species_array(species),
                                         len(species), _parr(Jn, n), _ptr(rho, n)))

    def num_tiles(self):
        return int(LIB.pic_num_tiles(self.h))

    def bin(self, species, offsets=None):
        arr = _species_array([species])
        self._check(LIB.pic_bin(self.h, arr, _ptr(offsets, self.num_tiles() + 1) if offsets is not None else None))

    def center_to_nodal(self, F, out):
        self._check(LIB.pic_center_to_nodal(self.h, _parr(F, self.ncell), _parr(out, self.ncell)))

    def center_to_yee(self, Jn, out):
        self._check(LIB.pic_center_to_yee(self.h, _parr(Jn, self.ncell), _parr(out, self.ncell)))

    def fft_forward(self, real, spec):
        self._check(LIB.pic_fft_forward(self.h, _parr(real, self.ncell), _parr(spec, 2 * self.nmode), len(real)))

    def fft_inverse(self, spec, real):
        self._check(LIB.pic_fft_inverse(self.h, _parr(spec, 2 * self.nmode), _parr(real, self.ncell), len(real)))

    def maxwell_step(self, E, B, J, rho_n, rho_np1, Eavg=None, Bavg=None):
        n = self.ncell
        ea = _parr(Eavg, n) if Eavg is not None else None
        ba = _parr(Bavg, n) if Bavg is not None else None
        self._check(LIB.pic_maxwell_step(self.h, _parr(E, n), _parr(B, n), _parr(J, n), _ptr(rho_n, n),
                                         _ptr(rho_np1, n), ea, ba))

    def coefficient(self, name, out):
        self._check(LIB.pic_coefficient(self.h, name.encode(), _ptr(out, 2 * self.nmode)))

    def field_energy(self, E, B, box_lo=None, box_hi=None):
        out = ctypes.c_double()
        lo = _l3(*box_lo) if box_lo is not None else None
        hi = _l3(*box_hi) if box_hi is not None else None
        self._check(LIB.pic_field_energy(self.h, _parr(E, self.ncell), _parr(B, self.ncell), lo, hi,
                                         ctypes.byref(out)))
        return out.value

    def total_charge(self, rho):
        out = ctypes.c_double()
        self._check(LIB.pic_total_charge(self.h, _ptr(rho, self.ncell), ctypes.byref(out)))
        return out.value

    def timing(self, enable):
        self._check(LIB.pic_timing(self.h, 1 if enable else 0))

    def timing_read(self, stage):
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        self._check(LIB.pic_timing_read(self.h, stage.encode(), ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    # ---- FP32 form ----
    def capture_step(self, E, B, J, rho, species, nsteps):
        """A CUDA graph of pic_step on these arrays (see StepGraph).  Runs the call once first."""
        return StepGraph(self, self.step, (E, B, J, rho, species, nsteps))

    def capture_step32(self, E, B, J, rho, species, nsteps):
        """A CUDA graph of pic_step32 on these arrays (see StepGraph).  Runs the call once first."""
        return StepGraph(self, self.step32, (E, B, J, rho, species, nsteps))

    def step32(self, E, B, J, rho, species, nsteps):
        n = self.ncell
        self._check(LIB.pic_step32(self.h, _parr(E, n), _parr(B, n), _parr(J, n) if J is not None else None,
                                   _ptr(rho, n),
                                   _species_array(species), len(species), nsteps))

    def deposit_rho32(self, species, rho):
        self._check(LIB.pic_deposit_rho32(self.h, _species_array(species), len(species), _ptr(rho, self.ncell)))

    def push_deposit32(self, En, Bn, species, Jn, rho):
        n = self.ncell
        self._check(LIB.pic_push_deposit32(self.h, _parr(En, n), _parr(Bn, n), _species_array(species),
                                           len(species), _parr(Jn, n), _ptr(rho, n)))

    def bin32(self, species, offsets=None):
        self._check(LIB.pic_bin32(self.h, _species_array([species]),
                                  _ptr(offsets, self.num_tiles() + 1) if offsets is not None else None))

    def fft_forward32(self, real, spec):
        self._check(LIB.pic_fft_forward32(self.h, _parr(real, self.ncell), _parr(spec, 2 * self.nmode), len(real)))

    def fft_inverse32(self, spec, real):
        self._check(LIB.pic_fft_inverse32(self.h, _parr(spec, 2 * self.nmode), _parr(real, self.ncell), len(real)))

    def field_energy32(self, E, B, box_lo=None, box_hi=None):
        out = ctypes.c_double()
        lo = _l3(*box_lo) if box_lo is not None else None
        hi = _l3(*box_hi) if box_hi is not None else None
        self._check(LIB.pic_field_energy32(self.h, _parr(E, self.ncell), _parr(B, self.ncell), lo, hi,
                                           ctypes.byref(out)))
        return out.value

    def total_charge32(self, rho):
        out = ctypes.c_double()
        self._check(LIB.pic_total_charge32(self.h, _ptr(rho, self.ncell), ctypes.byref(out)))
        return out.value

    def _ordered(self, fn, *args):
        """Call fn(ctx, *args) on the context's stream, ordered after the work already queued on
        torch's current stream (which made the inputs) and before the work queued there next."""
        cur = torch.cuda.current_stream()
        self.stream.wait_stream(cur)
        self._check(fn(self.h, *args))
        cur.wait_stream(self.stream)

    def species32_from_species(self, sp):
        """pic_species32_from_species: a new FP32-form species (device) from an FP64 one."""
        n = sp.n
        f = lambda: torch.empty(n, dtype=torch.float32, device="cuda")
        out = Species32(torch.empty(n, dtype=torch.int32, device="cuda"), f(), f(), f(), f(), f(), f(), f(),
                        sp.q, sp.m, id=torch.empty(n, dtype=torch.int64, device="cuda") if sp.id is not None else None)
        self._ordered(LIB.pic_species32_from_species, ctypes.byref(sp.c_struct()), ctypes.byref(out.c_struct()))
        return out

    def species32_to_species(self, sp32):
        """pic_species32_to_species: a new FP64 species (device) from an FP32-form one."""
        n = sp32.n
        f = lambda: torch.empty(n, dtype=torch.float64, device="cuda")
        out = Species(f(), f(), f(), f(), f(), f(), f(), sp32.q, sp32.m,
                      id=torch.empty(n, dtype=torch.int64, device="cuda") if sp32.id is not None else None)
        self._ordered(LIB.pic_species32_to_species, ctypes.byref(sp32.c_struct()), ctypes.byref(out.c_struct()))
        return out

    def field_energy_adjoint(self, E, B, box_lo, box_hi, scale, Ebar, Bbar):
        """pic_field_energy_adjoint: Ebar, Bbar (overwritten) = scale * dW/dE, dW/dB of the box."""
        n = self.ncell
        lo = _l3(*box_lo) if box_lo is not None else None
        hi = _l3(*box_hi) if box_hi is not None else None
        self._check(LIB.pic_field_energy_adjoint(self.h, _parr(E, n), _parr(B, n), lo, hi, float(scale),
                                                 _parr(Ebar, n), _parr(Bbar, n)))

    # ---- diagnostics (host results) ----
    def _axis_len(self, axis):
        return int(self.shape[axis]) if 0 <= axis < 3 else 1  # a bad axis is rejected by the library

    def stencil_extent(self, coef, axis):
        out = (ctypes.c_double * self._axis_len(axis))()
        self._check(LIB.pic_stencil_extent(self.h, coef.encode(), axis, out))
        return list(out)

    def axis_tables(self, axis):
        """([k]_s, [k]_c, zeta) along the axis, FFT order."""
        n = self._axis_len(axis)
        ks, kc, zt = (ctypes.c_double * n)(), (ctypes.c_double * n)(), (ctypes.c_double * n)()
        self._check(LIB.pic_axis_tables(self.h, axis, ks, kc, zt))
        return list(ks), list(kc), list(zt)

    def vacuum_dispersion(self, axis):
        out = (ctypes.c_double * self._axis_len(axis))()
        self._check(LIB.pic_vacuum_dispersion(self.h, axis, out))
        return list(out)

    def beam_rms(self, species):
        out = ctypes.c_double()
        self._check(LIB.pic_beam_rms(self.h, _species_array([species]), ctypes.byref(out)))
        return out.value

    def beam_rms32(self, species):
        out = ctypes.c_double()
        self._check(LIB.pic_beam_rms32(self.h, _species_array([species]), ctypes.byref(out)))
        return out.value

    # ---- reverse mode ----
    def adjoint_step(self, E, B, species, Ebar, Bbar, rhobar, species_bar):
        """pic_adjoint_step: species_bar is a list of dicts with tensors x, y, z, ux, uy, uz."""
        n = self.ncell
        arr = (PicSpeciesAdjoint * max(1, len(species_bar)))()
        for i, (s, b) in enumerate(zip(species, species_bar)):
            arr[i] = PicSpeciesAdjoint(s.n, *[_ptr(b[k], s.n) for k in ("x", "y", "z", "ux", "uy", "uz")])
        self._check(LIB.pic_adjoint_step(self.h, _parr(E, n), _parr(B, n), _species_array(species), len(species),
                                         _parr(Ebar, n), _parr(Bbar, n), _ptr(rhobar, n), arr))
