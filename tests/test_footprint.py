"""The paper's footprint and occupancy arithmetic against its printed tables
(Sec. 6.2, Tables 1-6, and the 4332-byte figure of Sec. 6.3.1)."""
import json
import os

from oracle import footprint as fp


def _tables(golden_dir):
    with open(os.path.join(golden_dir, "paper_tables.json")) as f:
        return json.load(f)


def test_table1_scalar_footprint(golden_dir):
    for n, stack, pre, tps, total in _tables(golden_dir)["table1_scalars_footprint"]["rows"]:
        assert fp.stack_scalars(n) == stack
        assert fp.prealloc_bytes() == pre and fp.THREAD_PRIVATE_BYTES == tps
        assert fp.footprint_scalars(n) == total


def test_table4_array_footprint(golden_dir):
    for k, stack, pre, tps, total in _tables(golden_dir)["table4_arrays_footprint"]["rows"]:
        assert fp.stack_arrays(k) == stack
        assert fp.footprint_arrays(k) == total


def _check_scalar_occupancy(rows, gpu):
    for n, smem, dyn, regs, teams, per_sm in rows:
        assert fp.footprint_scalars(n) == smem
        assert fp.global_list_bytes(n) == dyn
        assert fp.teams_by_registers(gpu, regs) == teams
        assert fp.smem_per_sm(teams, smem) == per_sm


def test_table2_k40(golden_dir):
    _check_scalar_occupancy(_tables(golden_dir)["table2_scalars_k40"]["rows"], fp.K40)


def test_table2b_p100(golden_dir):
    _check_scalar_occupancy(_tables(golden_dir)["table2b_scalars_p100"]["rows"], fp.P100)


def _check_array_occupancy(rows, gpu):
    for k, arr, smem, regs, pot, per_sm, actual in rows:
        assert 384 * k == arr
        assert fp.footprint_arrays(k) == smem
        assert fp.teams_by_registers(gpu, regs) == pot
        assert fp.smem_per_sm(pot, smem) == per_sm
        assert fp.teams_actual(gpu, regs, smem) == actual


def test_table5_k40(golden_dir):
    _check_array_occupancy(_tables(golden_dir)["table5_arrays_k40"]["rows"], fp.K40)


def test_table6_p100(golden_dir):
    _check_array_occupancy(_tables(golden_dir)["table6_arrays_p100"]["rows"], fp.P100)


def test_table3_register_row(golden_dir):
    for teams, regs in _tables(golden_dir)["table3_register_row_k40"]["rows"]:
        assert min(255, fp.REGS_PER_SM // (fp.TEAM_THREADS * teams)) == regs


def test_peak_k40_figure(golden_dir):
    d = _tables(golden_dir)["discussion_peak_k40"]
    teams = fp.teams_by_registers(fp.K40, d["registers"])
    assert teams == d["teams_per_sm"]
    total = fp.smem_per_sm(teams, fp.footprint_scalars(d["n_vars"]))
    assert total == d["smem_per_sm"]
    assert round(100 * total / fp.K40.smem_per_sm) == d["fraction_of_16k_percent"]
