"""CPU oracle for the inter-block synchronization workloads.  TEST INFRASTRUCTURE ONLY.

Only the tests, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py` may import,
call, link or run anything in this package.  The CUDA library never routes through it, and
it shares no code with the CUDA path: the two meet only in the seeded input arrays that the
callers pass to both.

Parts (each cites the paper passage it follows):
  calc        exact final states of each workload, written as their plain definitions.
  model_check explicit-state model checker that runs each primitive's algorithm as a
              per-block step machine and checks mutual exclusion, capacity, FIFO order,
              barrier safety and freedom from deadlock on tiny inputs.
  classify    the machine-abstraction arithmetic of Section 3 and Section 4 (Table 1 ->
              Tables 2 and 3 -> the three abstraction parameters -> a design choice).
  cpu         ctypes binding of cpu_exec.c, a threaded C program that executes the same
              workloads with real locks on host threads (C11 atomics); its final states are
              checked against `calc`, and its throughput is the CPU baseline.
"""
