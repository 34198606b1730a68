"""CPU-side checks of the C ABI: the library loads, exports every function that
include/dmrg_gb300.h declares, and rejects invalid problems before touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from workloads import hubbard_chain, random_integrals, round_robin_irreps

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dmrg_gb300.h")
LIB = os.path.join(ROOT, "paper_1312_2415_gb300", "_build", "libdmrg_gb300.so")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        import __graft_entry__
        __graft_entry__.build()
    from paper_1312_2415_gb300 import binding
    return binding.load(LIB)


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dmrg_[a-z_0-9]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 16
    raw = ctypes.CDLL(LIB)
    for n in names:
        assert hasattr(raw, n), n
    from paper_1312_2415_gb300.binding import EXPORTED
    assert set(EXPORTED) == set(names)


def test_invalid_problems_are_rejected(lib):
    from paper_1312_2415_gb300 import Context, DMRGError
    bad = [
        dict(L=4, orb_irrep=[0] * 4, N=1, two_S=1, target_irrep=0),   # N < 2 (Eq. 11)
        dict(L=4, orb_irrep=[0] * 4, N=9, two_S=1, target_irrep=0),   # N > 2L
        dict(L=4, orb_irrep=[0] * 4, N=4, two_S=1, target_irrep=0),   # parity of N - 2S
        dict(L=4, orb_irrep=[0] * 4, N=4, two_S=6, target_irrep=0),   # S > N/2
        dict(L=4, orb_irrep=[0, 1, 2, 3], N=4, two_S=0, target_irrep=5, group=4),  # irrep
        dict(L=4, orb_irrep=[0, 9, 0, 0], N=4, two_S=0, target_irrep=0, group=7),
    ]
    for kw in bad:
        with pytest.raises(DMRGError) as e:
            Context(**kw)
        assert e.value.code == -1
    with pytest.raises(DMRGError):
        Context(4, [0] * 4, 4, 0, 0, precision=3)


def test_symmetry_violations_are_rejected(lib):
    from paper_1312_2415_gb300 import Context, DMRGError
    L = 4
    irr = round_robin_irreps(L, 4)
    h, V = random_integrals(irr, 3, n_irrep=4)
    ctx = Context(L, irr, 4, 0, 0, group=4)
    ctx.set_integrals(h, V)  # valid
    h2 = h.copy(); h2[0, 1] += 0.1
    V2 = V.copy(); V2[0, 1, 2, 3] += 0.1
    h3 = h.copy(); h3[0, 1] = h3[1, 0] = 0.3       # couples irreps 0 and 1
    V3 = V.copy()
    for idx in {(0, 0, 0, 1), (0, 0, 1, 0), (0, 1, 0, 0), (1, 0, 0, 0)}:
        V3[idx] = 0.2                                # irrep product != A
    for hh, VV in ((h2, V), (h, V2), (h3, V), (h, V3)):
        with pytest.raises(DMRGError) as e:
            ctx.set_integrals(hh, VV)
        assert e.value.code == -2


def test_device_calls_fail_cleanly_without_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1312_2415_gb300 import Context, DMRGError
    h, V = hubbard_chain(4)
    ctx = Context(4, [0] * 4, 4, 0, 0)
    ctx.set_integrals(h, V)
    with pytest.raises(DMRGError) as e:
        ctx.init_mps(1)
    assert e.value.code == -5


def test_rdm_and_excitation_calls_check_their_state(lib):
    """Without an MPS the RDM and excited-state calls are rejected cleanly (DMRG_EINVAL
    from the state check, or DMRG_ECUDA where there is no device to set up a stream on);
    the count of lower states starts at zero."""
    from paper_1312_2415_gb300 import Context, DMRGError
    h, V = hubbard_chain(4)
    ctx = Context(4, [0] * 4, 4, 0, 0)
    assert ctx.excitation_count() == 0
    with pytest.raises(DMRGError) as e:
        ctx.rdm()
    assert e.value.code in (-1, -5)
    ctx.set_integrals(h, V)
    with pytest.raises(DMRGError) as e:
        ctx.push_excitation(1.0)
    assert e.value.code in (-1, -5)
    assert ctx.excitation_count() == 0
