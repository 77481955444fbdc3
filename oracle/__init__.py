"""CPU oracle for the hybrid IPM / column-generation OT solver (float64).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this package.
The product library (``paper_2206_11009_gb300``) never imports, links or runs it, and this
package never imports the product library: the two share no code.  The only module both
sides may receive data from is the seeded input generator, which holds no solver arithmetic.

Parts
-----
* ``netsimplex``  O1: exact optimum by a plain primal network simplex (C, ``netsimplex.c``).
* ``brute``       O3: vertex enumeration, assignment by permutations, 1-D monotone coupling.
* ``pricing``     the pricing rule of Section 3.4 with the exact selection contract.
* ``ipm``         O2: a plain rendition of the sparse IPM iteration of Sections 3-4.
* ``certificate`` LP certificates: c-transform lower bound, feasibility, acyclicity.

Pins: every function here is checked in ``tests/test_oracle_*.py`` against something other
than itself (brute force, closed forms, LP duality, invariants stated in the paper).  The
IPM trajectory (iteration counts) is "parity unpinned": only its end result is pinned.
"""
