"""Host logic of bench.py that needs no GPU: the deposit-array choice and the fast push's
algorithmic byte count (CPU)."""
import sys
import types

import bench


class _FakeLib:
    """Records the precision setters bench.set_deposits calls."""

    def __init__(self):
        self.calls = []

    def set_deposit_precision(self, p):
        self.calls.append(("deposit", p))

    def set_charge_precision(self, p):
        self.calls.append(("charge", p))


def _fake_module():
    return types.SimpleNamespace(FP_FP32=1, FP_FP64=0)


def test_deposit_choices_set_the_array_types():
    F = _fake_module()
    expect = {"fp32": [], "fp64": [("deposit", 0)], "change": [("charge", 0)], "change64": [("deposit", 0)]}
    for choice, calls in expect.items():
        lib = _FakeLib()
        bench.set_deposits(types.SimpleNamespace(deposits=choice), lib, F)
        assert lib.calls == calls, choice


def test_default_deposits_are_the_charge_change(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    args = bench.parse()
    assert args.deposits == "change" and args.tune_seeds == 2
    monkeypatch.setattr(sys, "argv", ["bench.py", "--deposits", "fp32"])
    assert bench.parse().deposits == "fp32"


def test_fast_push_bytes_count_each_array_at_its_width():
    sizes = {"n_tets": 10, "n_edges": 20, "n_nodes": 5}
    # 52 B per particle, 128 B per tet record, each dG and Q entry read and written once
    assert bench.fast_kernel_bytes(100, sizes) == 100 * 52 + 10 * 128 + 2 * 4 * (20 + 5)
    assert bench.fast_kernel_bytes(100, sizes, 4, 8) == 100 * 52 + 10 * 128 + 2 * (4 * 20 + 8 * 5)
    assert bench.fast_kernel_bytes(100, sizes, 8) == 100 * 52 + 10 * 128 + 2 * 8 * (20 + 5)
