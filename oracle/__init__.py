"""CPU oracle for the column-oriented Datalog fixpoint — TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the GPU
library.

* ``oracle.oracle``: C++ semi-naive / naive evaluator over std::set
  (whole-program fixpoints).
* ``oracle.primitives``: plain numpy/Python statements of each step of one
  round (hash index, join count / scan / write, sort, unique, difference,
  merge) for step-by-step parity.
* ``oracle.mlp``: float64 forward / backward of the join-size network.
"""
