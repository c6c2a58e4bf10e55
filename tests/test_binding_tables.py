"""The batch tables the binding builds for sprot_estimate_batch, checked field by field against
the sprot_instance layout without a GPU (not gpu)."""
import numpy as np
import pytest
import torch

from paper_2502_06337_gb300 import binding as B


def _lists(m=37, seed=0):
    rng = np.random.default_rng(seed)
    ns = rng.integers(1, 500, m)
    Ps = [torch.zeros((int(n), 3)) for n in ns]
    Qs = [torch.zeros((int(n), 3)) for n in ns]
    prms = [B.make_params(grid=(0, 64, 256)[i % 3], angle_bins=90 + i, k=1 + i % 4, tau=0.01 * (i + 1),
                          nms_deg=0.5 * i, gate_window=i % 3 - 1, angle_window=i % 2) for i in range(m)]
    return ns, Ps, Qs, prms


def test_list_table_fields():
    ns, Ps, Qs, prms = _lists()
    labels = [torch.zeros(int(n), dtype=torch.int32) if i % 4 == 0 else None for i, n in enumerate(ns)]
    tab, rot, nf, kmax = B._instance_table([(P, Q, p, L) for P, Q, p, L in zip(Ps, Qs, prms, labels)])
    assert kmax == max(p.k for p in prms) and rot.shape == (len(ns) * kmax,)
    for i in range(len(ns)):
        assert tab["P"][i] == Ps[i].data_ptr() and tab["Q"][i] == Qs[i].data_ptr() and tab["n"][i] == ns[i]
        assert tab["labels"][i] == (labels[i].data_ptr() if labels[i] is not None else 0)
        for name, _ in B.Params._fields_:
            assert tab["params." + name][i] == np.asarray(getattr(prms[i], name), tab["params." + name].dtype)
        assert tab["out"][i] == rot.ctypes.data + i * kmax * B.C.sizeof(B.Rotation)
        assert tab["n_found"][i] == nf.ctypes.data + 4 * i


def test_list_table_rejects_bad_points():
    ns, Ps, Qs, prms = _lists(m=3)
    with pytest.raises((AssertionError, ValueError)):
        B._instance_table([(Ps[0], Qs[1] if ns[0] != ns[1] else Qs[0][:-1], prms[0])])
    with pytest.raises((AssertionError, ValueError)):
        B._instance_table([(Ps[0].double(), Qs[0].double(), prms[0])])


def test_packed_table_fields():
    ns, Ps, Qs, prms = _lists()
    off = np.concatenate([[0], np.cumsum(ns)])
    P, Q = torch.cat(Ps), torch.cat(Qs)
    labels = torch.zeros(int(off[-1]), dtype=torch.int32)
    arr = B.params_array(len(ns), grid=[p.grid for p in prms], angle_bins=[p.angle_bins for p in prms],
                         k=[p.k for p in prms], tau=[p.tau for p in prms], nms_deg=[p.nms_deg for p in prms],
                         gate_window=[p.gate_window for p in prms], angle_window=[p.angle_window for p in prms])
    tab, rot, nf, kmax = B._packed_table(P, Q, off, arr, labels)
    ref, _, _, _ = B._instance_table([(P[off[i]:off[i + 1]], Q[off[i]:off[i + 1]], prms[i],
                                       labels[off[i]:off[i + 1]]) for i in range(len(ns))])
    for name in tab.dtype.names:
        if name not in ("out", "n_found"):
            assert np.array_equal(tab[name], ref[name]), name
    one, _, _, _ = B._packed_table(P, Q, off, B.make_params(grid=128, angle_bins=77, k=2))
    assert np.all(one["params.grid"] == 128) and np.all(one["params.angle_bins"] == 77) and np.all(one["params.k"] == 2)


@pytest.mark.parametrize("off", [[0, 5, 5, 10], [1, 10], [0, 9], [0, 11], [0]])
def test_packed_table_rejects_bad_offsets(off):
    P = torch.zeros((10, 3))
    with pytest.raises(ValueError):
        B._packed_table(P, P, off, B.make_params())
