"""The paper's static shared-memory footprint and occupancy arithmetic.

TEST INFRASTRUCTURE ONLY (part of the oracle). Restated from Sec. 6.2:

* Footprint per team (Sec. 6.2.1, Tables 1 and 4) = the shared stack
  allocated in the kernel prologue + the pre-allocated list of references
  (20 entries x 8 bytes = 160 B, Sec. 5.2) + the thread-private state kept
  in shared memory (49 B in these programs).
  - The shared depot mirrors the local depot (Sec. 5.3), one 8-byte slot per
    local; with n shared scalars there are two more locals, the team and
    thread numbers passed to the parallel call (Sec. 6.2.1), so the stack is
    8 (n + 2) bytes.
  - With k shared int[96] arrays the stack holds 384 B per array plus three
    8-byte slots: 24 + 384 k bytes.
* Teams per SM (Sec. 6.2.2, Tables 2, 2b, 5, 6): the register file (65536
  32-bit registers per SM) divided by 128 threads x registers per thread,
  capped by the concurrent-block limit (16 on K40, 32 on P100) and, for the
  "actual" column, by the shared memory per SM divided by the footprint.
* Shared memory per SM = teams per SM x footprint.
* When more than 20 references are shared, the list moves to global memory
  (Sec. 5.2, last paragraph): 8 bytes per shared variable (Tables 2, 2b).
"""
from __future__ import annotations

from dataclasses import dataclass

PREALLOC_ENTRIES = 20
PTR_BYTES = 8
THREAD_PRIVATE_BYTES = 49
REGS_PER_SM = 65536
TEAM_THREADS = 128


@dataclass(frozen=True)
class Gpu:
    name: str
    max_blocks_per_sm: int
    smem_per_sm: int


K40 = Gpu("K40", 16, 16 * 1024)   # default 16 KB shared / 48 KB L1 split
P100 = Gpu("P100", 32, 64 * 1024)


def prealloc_bytes() -> int:
    return PREALLOC_ENTRIES * PTR_BYTES


def stack_scalars(n_vars: int) -> int:
    return PTR_BYTES * (n_vars + 2)


def stack_arrays(n_arrays: int, elems: int = 96, elem_bytes: int = 4) -> int:
    return 3 * PTR_BYTES + n_arrays * elems * elem_bytes


def footprint_scalars(n_vars: int) -> int:
    return stack_scalars(n_vars) + prealloc_bytes() + THREAD_PRIVATE_BYTES


def footprint_arrays(n_arrays: int) -> int:
    return stack_arrays(n_arrays) + prealloc_bytes() + THREAD_PRIVATE_BYTES


def global_list_bytes(n_shared: int) -> int:
    return PTR_BYTES * n_shared if n_shared > PREALLOC_ENTRIES else 0


def teams_by_registers(gpu: Gpu, regs: int, threads: int = TEAM_THREADS) -> int:
    return min(gpu.max_blocks_per_sm, REGS_PER_SM // (threads * regs))


def teams_actual(gpu: Gpu, regs: int, footprint: int, threads: int = TEAM_THREADS) -> int:
    return min(teams_by_registers(gpu, regs, threads), gpu.smem_per_sm // footprint)


def smem_per_sm(teams: int, footprint: int) -> int:
    return teams * footprint
