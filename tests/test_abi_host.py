"""The C-ABI library without a GPU: it loads, exports every symbol include/kcm.h declares, and its
host-side construction (sample set, ZP geometry, links, bond classes) matches the oracle's
independent construction. Error paths return the documented codes."""
import os
import re

import numpy as np
import pytest

from oracle import oracle as O
from paper_1712_05012_b300 import kcm, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "kcm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kcm_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    import ctypes
    L = kcm.load()
    syms = declared_symbols()
    assert len(syms) >= 20
    for s in syms:
        assert hasattr(L, s), s
        assert ctypes.cast(getattr(L, s), ctypes.c_void_p).value
    assert set(syms) == set(kcm.EXPORTS)


@pytest.mark.parametrize("N", [1, 13, 256, 1000])
def test_sample_points_match_oracle(N):
    a = kcm.sample_points(N)
    b = O.sample_points(N)
    assert np.max(np.abs(a - b)) <= 2e-16


@pytest.mark.parametrize("m,seed", [(1, 3), (5, 4), (40, 1235)])
def test_zp_and_links_match_oracle(table, m, seed):
    seq = synth.sequence(m, seed)
    xyz, link = kcm.build_zp(seq, table, synth.GEOMETRY)
    ch = O.OracleChain(seq, table, synth.GEOMETRY)
    assert xyz.shape == (ch.n, 3)
    assert np.max(np.abs(xyz - ch.zp())) < 1e-12
    assert np.array_equal(link, ch.link)
    # defaults equal the generator's geometry
    xyz2, _ = kcm.build_zp(seq, table, None)
    assert np.max(np.abs(xyz2 - xyz)) < 1e-15


def test_pair_classes_match_oracle_bfs(table):
    m = 12
    seq = synth.sequence(m, 77)
    ch = O.OracleChain(seq, table, synth.GEOMETRY)
    a, b, want = [], [], []
    for i in range(ch.n):
        for j in range(i + 1, ch.n):
            if abs(ch.res[i] - ch.res[j]) <= 2:
                a.append(i)
                b.append(j)
                d = ch.bond_distance(i, j)
                want.append(1 if d <= 2 else (2 if d == 3 else 0))
    got = kcm.pair_class(seq, table, a, b)
    assert np.array_equal(got, np.array(want))
    assert (got == 2).sum() > 0 and (got == 1).sum() > 0


def test_natoms(table):
    seq = synth.sequence(33, 5)
    assert kcm.topology_natoms(seq, table) == synth.n_atoms(seq)


def test_error_paths(table):
    seq = synth.sequence(4, 1)
    with pytest.raises(kcm.KcmError) as e:
        kcm.Chain(seq, table, synth.RunParams(cutoff=-1.0))
    assert e.value.code == kcm.KCM_E_INVAL
    with pytest.raises(kcm.KcmError) as e:
        kcm.Chain(seq, table, synth.RunParams(n_sample=0))
    assert e.value.code == kcm.KCM_E_INVAL
    with pytest.raises(kcm.KcmError) as e:
        kcm.Chain(seq, table, synth.RunParams(side_joints=2))
    assert e.value.code == kcm.KCM_E_INVAL
    bad = seq.copy()
    bad[1] = 99
    with pytest.raises(kcm.KcmError) as e:
        kcm.topology_natoms(bad, table)
    assert e.value.code == kcm.KCM_E_INVAL


def test_create_without_device_fails_loudly(table):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    with pytest.raises(kcm.KcmError) as e:
        kcm.Chain(synth.sequence(4, 1), table, synth.RunParams())
    assert e.value.code == kcm.KCM_E_NODEVICE


def test_params_layout_and_defaults():
    """The binding's kcm_params has the C struct's size (eleven doubles, five int32, padded to 8) and
    kcm_params_default fills every field, the last one included."""
    import ctypes
    assert ctypes.sizeof(kcm.Params) == 112
    p = kcm.Params()
    for name, _ in kcm.Params._fields_:
        setattr(p, name, 7)
    assert kcm.load().kcm_params_default(ctypes.byref(p)) == kcm.KCM_OK
    d = synth.RunParams()
    for name, _ in kcm.Params._fields_:
        assert getattr(p, name) == getattr(d, name), name
