"""Host-side checks of the C ABI (no GPU needed): the library builds, loads and
exports every function declared in include/pic.h; the binding mirrors them."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pic.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pic_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("pic_init", "pic_step", "pic_destroy", "pic_field_energy", "pic_maxwell_step"):
        assert required in names


def test_library_exports_every_declared_symbol():
    import ctypes
    from paper_2106_12919_gb300 import build
    lib = ctypes.CDLL(build.build())
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    from paper_2106_12919_gb300 import pic
    assert sorted(pic.EXPORTS) == _declared()


def test_ext_defaults():
    import ctypes
    from paper_2106_12919_gb300 import pic
    e = pic.PicExt()
    pic.LIB.pic_ext_default(ctypes.byref(e))
    assert e.struct_size == ctypes.sizeof(pic.PicExt)
    assert (e.c, e.eps0, list(e.tile), e.sort_interval) == (1.0, 1.0, [8, 8, 8], 20)
    assert (e.filter_passes, e.pusher, e.cycle, e.reserved) == (0, pic.PIC_PUSHER_BORIS, pic.PIC_CYCLE_HYBRID, 0)


def test_init_rejects_bad_extension_fields():
    import ctypes
    from paper_2106_12919_gb300 import pic
    h = ctypes.c_void_p()
    L3, D3, I3 = ctypes.c_int64 * 3, ctypes.c_double * 3, ctypes.c_int32 * 3
    for field, value in (("filter_passes", 9), ("filter_passes", -1), ("pusher", 2), ("cycle", 4), ("reserved", 1)):
        e = pic.PicExt()
        pic.LIB.pic_ext_default(ctypes.byref(e))
        setattr(e, field, value)
        st = pic.LIB.pic_init(ctypes.byref(h), L3(16, 16, 16), D3(1, 1, 1), 1.0, 1, I3(8, 8, 8), 0, D3(0, 0, 0),
                              ctypes.byref(e))
        assert st == -1 and not h.value, field


def test_init_rejects_bad_arguments_without_gpu_work():
    """Validation happens before any device call: these return errors even without a GPU."""
    import ctypes
    from paper_2106_12919_gb300 import pic
    h = ctypes.c_void_p()
    L3, D3, I3 = ctypes.c_int64 * 3, ctypes.c_double * 3, ctypes.c_int32 * 3
    bad = [
        (L3(12, 16, 16), I3(8, 8, 8), 1, 0),      # not a power of two
        (L3(16, 16, 16), I3(7, 8, 8), 1, 0),      # odd centering order
        (L3(16, 16, 16), I3(8, 8, 8), 4, 0),      # shape order
        (L3(16, 16, 16), I3(8, 8, 8), 1, 5),      # variant
        (L3(16, 16, 8), I3(8, 8, 8), 1, 0),       # Nz < 16
    ]
    for grid, co, so, var in bad:
        st = pic.LIB.pic_init(ctypes.byref(h), grid, D3(1, 1, 1), 1.0, so, co, var, D3(0, 0, 0), None)
        assert st in (-1, -2)
        assert not h.value
    st = pic.LIB.pic_init(ctypes.byref(h), L3(16, 16, 16), D3(1, 1, 1), 1.0, 1, I3(8, 8, 8), 1, D3(0, 0, 1.5), None)
    assert st == -1                            # |v_gal| >= c


def test_fdtd_cycle_validation_without_gpu_work():
    """The FDTD cycle: the Galilean variants and a dt above its Courant limit are refused
    before any device call."""
    import ctypes
    from paper_2106_12919_gb300 import pic
    from oracle import fdtd
    L3, D3, I3 = ctypes.c_int64 * 3, ctypes.c_double * 3, ctypes.c_int32 * 3

    def init(dt, variant=0, dx=(1.0, 1.0, 1.0), orders=(0, 0, 0), **fields):
        h = ctypes.c_void_p()
        e = pic.PicExt()
        pic.LIB.pic_ext_default(ctypes.byref(e))
        e.cycle = pic.PIC_CYCLE_HYBRID_FDTD
        e.spectral_order[:] = list(orders)
        for k, v in fields.items():
            setattr(e, k, v)
        st = pic.LIB.pic_init(ctypes.byref(h), L3(16, 16, 16), D3(*dx), dt, 1, I3(8, 8, 8), variant,
                              D3(0, 0, 0.5), ctypes.byref(e))
        assert not h.value or st == 0
        return st

    assert init(0.5, variant=1) == -2                    # Galilean
    assert init(0.5, variant=2) == -2                    # averaged Galilean
    # difference order above 32 (the host weight table's size), refused before any device work
    h = ctypes.c_void_p()
    e = pic.PicExt()
    pic.LIB.pic_ext_default(ctypes.byref(e))
    e.cycle = pic.PIC_CYCLE_HYBRID_FDTD
    e.spectral_order[:] = [2, 2, 64]
    st = pic.LIB.pic_init(ctypes.byref(h), L3(16, 16, 128), D3(1, 1, 1), 0.01, 1, I3(8, 8, 8), 0, D3(0, 0, 0),
                          ctypes.byref(e))
    assert st == -1 and not h.value
    for dx, orders in (((1.0, 1.0, 1.0), (0, 0, 0)), ((0.2, 0.2, 0.04), (4, 4, 8)), ((1.0, 0.5, 2.0), (2, 6, 4))):
        lim = fdtd.courant_limit(tuple(o or 2 for o in orders), dx)
        assert init(lim * 1.001, dx=dx, orders=orders) == -1, (dx, orders)


def test_centering_rejects_overlapping_arrays_without_gpu_work():
    """pic_center_to_nodal_static refuses outputs that overlap an input or another output before
    any device call (the stencil passes cannot run in place).  The addresses are never used."""
    import ctypes
    from paper_2106_12919_gb300 import pic
    L3, I3, P6 = ctypes.c_int64 * 3, ctypes.c_int32 * 3, ctypes.c_void_p * 6
    ncell = 8 * 8 * 16
    nbytes = ncell * 8
    base = 1 << 40
    F = P6(*[base + c * nbytes for c in range(6)])
    outs = [base + (6 + c) * nbytes for c in range(6)]
    cases = {"in place": 0, "into a later input": 3 * nbytes, "half overlap": nbytes // 2}
    for what, off in cases.items():
        o = list(outs)
        o[2] = base + off
        st = pic.LIB.pic_center_to_nodal_static(L3(8, 8, 16), I3(4, 4, 4), F, P6(*o), None)
        assert st == -1, what
    o = list(outs)
    o[4] = o[1]
    assert pic.LIB.pic_center_to_nodal_static(L3(8, 8, 16), I3(4, 4, 4), F, P6(*o), None) == -1
