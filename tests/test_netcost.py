"""The core kernel's counted work (its ALU roofline's numerator), CPU only.

The counts come from the generated selection networks; the per-request work
adds the sparse items by how the kernel decides them (the network, or a rank
test of one comparison per window value).  These checks tie the numbers the
benchmark divides by to the networks and to the documented formula.
"""
import pytest

from paper_2602_17938_gb300 import netcost


def test_network_counts():
    c = netcost.counts()
    assert c["med5x5"] == 188 and c["med7x7"] == 586 and c["med3x3"] == 38
    assert c["dense_med5_per_px"] == pytest.approx(73.5)   # 4x2 block: 588 ops for 8 outputs
    assert c["dense_med3_per_px"] == pytest.approx(17.25)  # 8x2 block: 276 ops for 16 outputs


def test_detect_work_formula():
    prof = {"px_iterations": 10_000, "px_core": 8_000, "n_sprime": 1_000, "n_sprime_net": 100,
            "n_fine": 90, "n_fine_net": 4}
    w = netcost.detect_work(prof, packed=True)
    dense = 8_000 * (73.5 + 17.25)
    assert w["dense_elem"] == pytest.approx(dense)
    assert w["dense_instr"] == pytest.approx(dense / 2)  # one u16x2 instruction per two outputs
    assert w["sprime_instr"] == 100 * 188 + 900 * netcost.RANK_TEST_LO
    assert w["fine_instr"] == 4 * 586 + 86 * netcost.RANK_TEST_OBJLIM
    assert w["instr"] == pytest.approx(dense / 2 + w["sprime_instr"] + w["fine_instr"])
    assert w["instr_as_networks"] == pytest.approx(dense / 2 + 1_000 * 188 + 90 * 586)
    assert netcost.RANK_TEST_LO == 25 and netcost.RANK_TEST_OBJLIM == 49
    # float32 frames: no packing
    assert netcost.detect_work(prof, packed=False)["dense_instr"] == pytest.approx(dense)


def test_profiles_without_network_counters_count_every_median_as_a_network():
    prof = {"px_iterations": 100, "n_sprime": 10, "n_fine": 3}
    w = netcost.detect_work(prof, packed=False)
    assert w["sprime_instr"] == 10 * 188 and w["fine_instr"] == 3 * 586
    assert w["instr"] == pytest.approx(w["instr_as_networks"])
