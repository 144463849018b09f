"""The C ABI library builds, loads without a GPU and exports every declared symbol."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"\b(vlasov_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    from paper_2110_15867_gb300 import binding, build
    build.build()
    lib = ctypes.CDLL(build.LIB)
    decl = declared_symbols()
    assert len(decl) >= 9
    missing = [s for s in decl if not hasattr(lib, s)]
    assert not missing, missing
    assert set(binding.SYMBOLS) <= set(decl)


def test_init_rejects_bad_grids_without_touching_the_gpu():
    from paper_2110_15867_gb300 import binding as B
    B.load(build_if_missing=True)
    g = B.Grid()
    g.nx, g.ny, g.nz, g.nux, g.nuy, g.nuz = 8, 8, 8, 6, 8, 8  # 6 is not a multiple of 4
    g.L, g.V, g.dtype = 1.0, 5.0, B.F32
    with pytest.raises(B.VlasovError) as e:
        B.vlasov_init(g, 16, None, 0)
    assert e.value.code == B.EINVAL
    g.nux = 8
    with pytest.raises(B.VlasovError) as e:
        B.vlasov_init(g, 8, None, 0)  # misaligned pointer
    assert e.value.code == B.EINVAL
    with pytest.raises(B.VlasovError):
        B.vlasov_init(g, 0, None, 0)


@pytest.mark.parametrize("field,value", [("nx", 0), ("nz", 3), ("nuz", 0), ("nuy", 2), ("V", 0.0), ("L", -1.0),
                                         ("dtype", 7)])
def test_init_rejects_empty_and_degenerate_grids(field, value):
    # an empty grid (a zero extent), lines too short for the five-cell stencil, a
    # non-positive box or velocity bound and an unknown storage type are refused on the
    # host with EINVAL, before any device call
    from paper_2110_15867_gb300 import binding as B
    B.load(build_if_missing=True)
    g = B.Grid()
    g.nx, g.ny, g.nz, g.nux, g.nuy, g.nuz = 8, 8, 8, 8, 8, 8
    g.L, g.V, g.dtype = 1.0, 5.0, B.F32
    setattr(g, field, value)
    with pytest.raises(B.VlasovError) as e:
        B.vlasov_init(g, 16, None, 0)
    assert e.value.code == B.EINVAL


def test_codec_rejects_bad_arguments_without_touching_the_gpu():
    # vlasov_encode / vlasov_decode check sizes, types and pointers on the host first;
    # nothing to do (zero lines) returns at once
    from paper_2110_15867_gb300 import binding as B
    B.load(build_if_missing=True)
    bad = [(4, 0, 16, B.F64, 16, B.BF16, 16), (4, 129, 16, B.F64, 16, B.BF16, 16),
           (-1, 16, 16, B.F64, 16, B.BF16, 16), (4, 16, 16, B.BF16, 16, B.BF16, 16),
           (4, 16, 16, B.F64, 16, B.F32, 16), (4, 16, None, B.F64, 16, B.BF16, 16),
           (4, 16, 12, B.F64, 16, B.BF16, 16), (4, 16, 16, B.F32, 17, B.F16, 16),
           (4, 16, 16, B.F32, 16, B.F16, 18)]
    for nl, nuz, src, sdt, codes, cdt, scale in bad:
        with pytest.raises(B.VlasovError) as e:
            B.vlasov_encode(nl, nuz, src, sdt, codes, cdt, scale, 0)
        assert e.value.code == B.EINVAL
        with pytest.raises(B.VlasovError) as e:
            B.vlasov_decode(nl, nuz, codes, cdt, scale, src, sdt, 0)
        assert e.value.code == B.EINVAL
    assert B.vlasov_encode(0, 16, None, B.F64, None, B.BF16, None, 0) == B.OK
    assert B.vlasov_decode(0, 16, None, B.BF16, None, None, B.F32, 0) == B.OK
