"""The C ABI library on the CPU: it loads, exports every entry point the
headers declare, and its host-side checks behave (no kernel launches)."""
import os
import re

import pytest

import paper_1711_10413_gb300 as dsr
import workloads as wl
from paper_1711_10413_gb300 import builder as dsr_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    dsr_build.build()
    return dsr.lib()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(dsr_\w+)\s*\(", text, re.M))
    return names


def test_exports_every_declared_symbol(L):
    declared = _declared()
    assert "dsr_launch_region" in declared and len(declared) >= 9
    for name in declared:
        assert hasattr(L, name), name


def test_binding_covers_declared_symbols(L):
    assert _declared() <= set(dsr.exported_symbols())


def test_validate_and_extent(L):
    w = wl.nested(teams=8, threads=256, depth=3)
    r = w.regions[0]
    ib, ob, ns = dsr.dsr_region_extent(r)
    assert (ib, ob, ns) == (8 * 3 * 1088, 4 * 8 * 4096, 8)
    assert dsr.dsr_validate_region(r, ib, ob, ns) == dsr.DSR_OK
    assert dsr.dsr_validate_region(r, ib - 1, ob, ns) == dsr.DSR_ERR_INVALID
    assert dsr.dsr_validate_region(r, ib, ob, ns - 1) == dsr.DSR_ERR_INVALID
    bad = [
        dict(r.as_dict(), frame_bytes=[1088, 1088, 1000, 0]),
        dict(r.as_dict(), threads=100),
        dict(r.as_dict(), threads=2048),
        dict(r.as_dict(), depth=5),
        dict(r.as_dict(), width=300),
        dict(r.as_dict(), image_offset=8),
        dict(r.as_dict(), program=42),
        dict(r.as_dict(), teams=0),
    ]
    for b in bad:
        assert dsr.dsr_validate_region(b, 1 << 40, 1 << 40, 1 << 30) == dsr.DSR_ERR_INVALID, b
        assert dsr.dsr_last_error_string(None), b  # each rejection says why


def test_extent_matches_workloads(L):
    for work in [wl.paper_scalars(7), wl.paper_arrays(3), wl.scalars(100),
                 wl.sweep(8192, teams=4), wl.hetero(30, max_teams=4)]:
        for r in work.regions:
            ib, ob, ns = dsr.dsr_region_extent(r)
            assert r.image_offset + ib <= work.images.size
            assert r.out_offset + ob <= work.out_bytes
            assert r.status_index + ns <= work.n_status
            assert dsr.dsr_validate_region(r, work.images.size, work.out_bytes,
                                           work.n_status) == 0


def test_footprint_model(L):
    r = wl.nested(teams=1024, threads=256, depth=3).regions[0]
    f = dsr.dsr_footprint_model(r, slab_bytes=3264, regs=32)
    assert f["smem_per_team"] == f["ctrl_bytes"] + 3264 and f["spill_bytes"] == 0
    assert f["teams_per_sm"] == 8 and f["limit"] == 1          # 64 warps / 8
    f = dsr.dsr_footprint_model(r, slab_bytes=2176, regs=32)
    assert f["spill_bytes"] == 1088                           # third frame spills
    s = wl.sweep(196608, teams=512).regions[0]
    f = dsr.dsr_footprint_model(s, slab_bytes=196608, regs=32)
    assert f["teams_per_sm"] == 1 and f["limit"] == 2          # 192 KiB slab
    f = dsr.dsr_footprint_model(s, slab_bytes=0, regs=32)
    assert f["spill_bytes"] == 196608 and f["teams_per_sm"] == 16
    with pytest.raises(dsr.DsrError):
        dsr.dsr_footprint_model(s, slab_bytes=240000)


def test_create_without_gpu_fails_cleanly(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(dsr.DsrError) as ei:
        dsr.dsr_create(0)
    assert ei.value.code == dsr.DSR_ERR_CUDA
    assert "CUDA" in dsr.dsr_last_error_string(None) or "device" in dsr.dsr_last_error_string(None)


def test_occupancy_rejects_missing_context(L):
    # the occupancy query needs a context with a stack configuration; its
    # argument checks run before any CUDA call
    r = wl.nested(teams=8, threads=256, depth=3).regions[0]
    with pytest.raises(dsr.DsrError) as ei:
        dsr.dsr_region_occupancy(None, r)
    assert ei.value.code == dsr.DSR_ERR_INVALID


def _oracle_rows(work, i, slab, ovf):
    import oracle
    _, st = oracle.run_workload(work, slab_bytes=slab, overflow_bytes=ovf, regions=[i])
    r = work.regions[i]
    return st[r.status_index: r.status_index + r.teams]


def _footprint_cases():
    cases = [wl.paper_scalars(7, teams=2), wl.paper_scalars(40, teams=2, threads=64),
             wl.paper_arrays(3, teams=2), wl.scalars(5, teams=2),
             wl.hetero(25, max_teams=3, max_frame=4096)]
    cases += [wl.nested(teams=2, threads=128, depth=d, elems_per_team=8) for d in (1, 2, 3, 4)]
    cases += [wl.sweep(S, teams=2) for S in (4, 20, 1092, 8192)]
    cases += [wl.workers(teams=2, threads=t, frame_bytes=S, width=w)
              for t, S, w in [(64, 64, 0), (256, 100, 0), (160, 36, 45), (96, 4, 1), (1024, 20, 0)]]
    return cases


def test_region_footprint_matches_the_oracles_stack(L):
    """The library's footprint estimate (host code, from the descriptor
    alone) against the oracle's stack accounting: the peak stack bytes equal
    the hwm a team reports, and the slab estimate is tight -- with it
    nothing spills, with 16 bytes less something does."""
    for work in _footprint_cases():
        for i, r in enumerate(work.regions):
            stack, slab = dsr.dsr_region_footprint(r)
            assert slab % 16 == 0 and slab >= stack
            rows = _oracle_rows(work, i, 1 << 40, 0)
            assert (rows["status"] == 0).all()
            assert (rows["hwm_bytes"] == stack).all(), (work.name, r)
            rows = _oracle_rows(work, i, slab, 1 << 30)
            assert (rows["status"] == 0).all() and (rows["spill_bytes"] == 0).all()
            rows = _oracle_rows(work, i, slab - 16, 1 << 30)
            assert (rows["status"] == 0).all() and (rows["spill_bytes"] > 0).all(), (work.name, r)


def test_footprint_model_spill_matches_the_oracle(L):
    """dsr_footprint_model's bytes per team left to the overflow slab, for a
    slab between nothing and everything, against the oracle's spill."""
    for work in _footprint_cases():
        for i, r in enumerate(work.regions):
            _, slab = dsr.dsr_region_footprint(r)
            for sl in {0, 16, slab // 2 // 16 * 16, slab - 16, slab}:
                if sl + 384 > 232448:
                    continue
                model = dsr.dsr_footprint_model(r, sl, 32)["spill_bytes"]
                rows = _oracle_rows(work, i, sl, 1 << 30)
                assert (rows["spill_bytes"] == model).all(), (work.name, r, sl)


def test_bounded_wait_check_rejects_missing_context(L):
    """Checked on the host before anything launches."""
    assert L.dsr_check_bounded_wait(None, 1000, None, None) == dsr.DSR_ERR_INVALID


def test_stack_check_rejects_bad_arguments(L):
    assert L.dsr_check_stack(None, None, 0, None, 0, None) == dsr.DSR_ERR_INVALID


def test_report_error_records_the_message(L):
    """dsr_report_error: the way code built on the library (the launch
    templates of dsr_device.cuh) reports a failure; no ctx needed."""
    assert dsr.dsr_report_error(None, dsr.DSR_ERR_BUDGET, "pool too small for x") == 4
    assert dsr.lib().dsr_last_error_string(None).decode() == "pool too small for x"


def test_user_program_library_builds_and_exports(L):
    """A program written against include/dsr_device.cuh compiles (nvcc,
    sm_103a) into its own library linked with libdsr, exporting the test
    programs' entry points; descriptors naming a user program id pass the
    host-side shape check with no extent of their own."""
    import ctypes
    src = os.path.join(ROOT, "tests", "user_program", "user_programs.cu")
    out = os.path.join(ROOT, "tests", "user_program", "libuser_programs.so")
    dsr_build.build_user([src], out)
    U = ctypes.CDLL(out)
    for name in ("user_paper_scalars", "user_hetero"):
        for suffix in ("_launch", "_launch_batch", "_serve_start", "_serve_program",
                       "_program"):
            assert hasattr(U, name + suffix)
    U.user_hetero_program.restype = ctypes.c_uint32
    assert U.user_hetero_program() == dsr.DSR_PROG_USER + 6
    r = wl.hetero(n_instances=1, max_teams=4, max_frame=256).regions[0]
    r.program = dsr.DSR_PROG_USER + 6
    assert dsr.dsr_region_extent(r) == (0, 0, r.teams)
    r.program = 200   # neither built in nor in the user range
    with pytest.raises(dsr.DsrError):
        dsr.dsr_region_extent(r)


def test_user_server_hooks_check_descriptors(L):
    """The hook table a user program's server hands the library: its id, and
    a descriptor check (host code, run here) that passes well-formed
    requests inside the server's buffers and refuses the rest; the start
    call refuses a missing ctx or table without touching a GPU."""
    import ctypes
    src = os.path.join(ROOT, "tests", "user_program", "user_programs.cu")
    out = os.path.join(ROOT, "tests", "user_program", "libuser_programs.so")
    dsr_build.build_user([src], out)
    U = ctypes.CDLL(out)
    U.user_hetero_serve_program.restype = ctypes.POINTER(dsr.dsr_serve_program)
    prog = U.user_hetero_serve_program().contents
    assert prog.program == dsr.DSR_PROG_USER + 6 and prog.reserved == 0
    assert prog.validate and prog.prepare and prog.launch
    work = wl.hetero(n_instances=6, max_teams=4, max_frame=2048, seed=4)
    ib = work.images.nbytes
    ob = work.out_bytes
    ns = work.n_status
    for r in work.regions:
        r.program = dsr.DSR_PROG_USER + 6
        d = dsr.pack_desc(r)
        assert prog.validate(ctypes.addressof(d), ib, ob, ns) == dsr.DSR_OK
        # outputs, images or statuses one short of what the region indexes
        end_out = r.out_offset + 4 * r.teams * (r.width or max(r.threads - 32, 1))
        assert prog.validate(ctypes.addressof(d), ib, end_out - 4, ns) == dsr.DSR_ERR_INVALID
        assert prog.validate(ctypes.addressof(d), ib, ob, r.status_index + r.teams - 1) == \
            dsr.DSR_ERR_INVALID
        d.program = dsr.DSR_PROG_HETERO   # another program's descriptor
        assert prog.validate(ctypes.addressof(d), ib, ob, ns) == dsr.DSR_ERR_INVALID
    cfg = dsr.dsr_serve_cfg()
    cfg.program = prog.program
    assert dsr.lib().dsr_serve_start_user(None, ctypes.byref(cfg), None, 0,
                                          ctypes.byref(prog)) == dsr.DSR_ERR_INVALID
    assert dsr.lib().dsr_serve_start_user(None, ctypes.byref(cfg), None, 0, None) == \
        dsr.DSR_ERR_INVALID


def test_batch_abort_and_progress_refuse_without_ctx(L):
    """Host-side refusals of the abort and progress calls (no GPU touched)."""
    import ctypes
    assert dsr.lib().dsr_batch_abort(None, None) == dsr.DSR_ERR_INVALID
    t = ctypes.c_uint64()
    assert dsr.lib().dsr_batch_progress(None, None, ctypes.byref(t), None, None) == \
        dsr.DSR_ERR_INVALID


def test_graph_calls_refuse_without_ctx(L):
    """Host-side refusals of the launch-graph calls (no GPU touched)."""
    import ctypes
    g = ctypes.c_void_p()
    assert dsr.lib().dsr_graph_capture_regions(None, None, None, 0, ctypes.byref(g)) == \
        dsr.DSR_ERR_INVALID
    assert dsr.lib().dsr_graph_launch(None, None, None) == dsr.DSR_ERR_INVALID
    assert dsr.lib().dsr_graph_destroy(None) == dsr.DSR_OK
