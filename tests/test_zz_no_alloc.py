"""kcm_torques_noalloc: the torque entry point for callers that cannot allocate device memory
(for example a server whose GPU memory is all reserved by its own pool allocator). It keeps its
working memory in a fixed array inside the library, so these tests check that two calls in a row,
sharing that array, each give the torques of the regular kcm_torques entry point, and that sizes
beyond the array's limit are refused. This file is collected last on purpose."""
import numpy as np
import pytest

from kcm_testutil import Index, rel_inf
from oracle import oracle as O
from paper_1712_05012_b300 import synth

pytestmark = pytest.mark.gpu
TOL_FP64 = 1e-10  # the FP64 torque bar of the parity tests


def case(kcm, table, m, seed, solvation=1):
    """Positions, forces and torques of one chain from the regular entry points, plus the inputs
    the no-allocation call needs (link ranges, current joint axes and axis points), at a compact
    start. (An extended start of 16,000 residues puts atoms 57,000 A from the origin, and the two
    entry points' different summation orders then differ by 2e-10 of the largest torque.)"""
    seq = synth.sequence(m, seed)
    theta = synth.theta_from_codes(O.OracleChain(seq, table, synth.GEOMETRY).grow_start(seed))
    p = synth.RunParams(precision=synth.PRECISION_FP64, solvation=solvation)
    with kcm.Chain(seq, table, p) as ch:
        ch.set_theta(theta)
        xyz = ch.positions()
        F = ch.forces()
        tau = ch.torques()
    _, link = kcm.build_zp(seq, table)
    L = 2 * m + 1
    link_start = np.searchsorted(link, np.arange(L + 1)).astype(np.int32)
    ix = Index(seq)
    axis = np.zeros((2 * m, 3))
    point = np.zeros((2 * m, 3))
    for i in range(m):
        for j, (a, b) in enumerate(((ix.N(i), ix.CA(i)), (ix.CA(i), ix.C(i)))):
            d = xyz[b] - xyz[a]
            axis[2 * i + j] = d / np.linalg.norm(d)
            point[2 * i + j] = xyz[a]
    return dict(L=L, link_start=link_start, xyz=xyz, F=F, axis=axis, point=point, tau=tau)


def run_noalloc(kcm, c):
    import torch
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    ls, x, f, u, p = dev(c["link_start"]), dev(c["xyz"]), dev(c["F"]), dev(c["axis"]), dev(c["point"])
    tau = torch.full((c["L"] - 1,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    kcm.torques_noalloc(c["L"], ls.data_ptr(), x.data_ptr(), f.data_ptr(), u.data_ptr(), p.data_ptr(),
                        tau.data_ptr(), stream)
    torch.cuda.synchronize()
    return tau.cpu().numpy()


def test_two_calls_in_a_row_match_kcm_torques(table):
    from paper_1712_05012_b300 import kcm
    a = case(kcm, table, 120, 31)  # a larger chain first ...
    b = case(kcm, table, 17, 32)   # ... then a smaller one, which reuses the shared scratch
    ta = run_noalloc(kcm, a)
    tb = run_noalloc(kcm, b)
    assert rel_inf(ta, a["tau"]) < TOL_FP64
    assert rel_inf(tb, b["tau"]) < TOL_FP64


def test_largest_and_chunked_sizes(table):
    """The sizes that stress the fixed array: L = KCM_NOALLOC_MAX_LINKS exactly (16,383 residues and one
    empty link: the chunk sums fill their part of the array to the last word, and each scan thread takes
    64 chunks),
    then L = 601, where scan threads take more than one chunk, reusing what the larger call left."""
    from paper_1712_05012_b300 import kcm
    big = case(kcm, table, (kcm.NOALLOC_MAX_LINKS - 1) // 2, 33, solvation=0)
    # a chain has L = 2m + 1 links (odd): one more link without atoms reaches the limit exactly; its
    # joint moves nothing, so its torque is 0 and every other joint's is unchanged
    assert big["L"] == kcm.NOALLOC_MAX_LINKS - 1
    big["L"] += 1
    big["link_start"] = np.append(big["link_start"], big["link_start"][-1]).astype(np.int32)
    big["axis"] = np.vstack([big["axis"], [0.0, 0.0, 1.0]])
    big["point"] = np.vstack([big["point"], [1.0, 2.0, 3.0]])
    big["tau"] = np.append(big["tau"], 0.0)
    mid = case(kcm, table, 300, 34)
    assert mid["L"] == 601
    assert rel_inf(run_noalloc(kcm, big), big["tau"]) < TOL_FP64
    assert rel_inf(run_noalloc(kcm, mid), mid["tau"]) < TOL_FP64


def test_size_limit_is_refused(table):
    from paper_1712_05012_b300 import kcm
    import torch
    t = torch.zeros(8, dtype=torch.float64, device="cuda")
    ptr = t.data_ptr()
    with pytest.raises(kcm.KcmError) as e:
        kcm.torques_noalloc(kcm.NOALLOC_MAX_LINKS + 1, ptr, ptr, ptr, ptr, ptr, ptr)
    assert e.value.code == kcm.KCM_E_INVAL
