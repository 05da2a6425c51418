"""FP64 CPU oracle of the joint lensing + dynamics log-likelihood.

TEST INFRASTRUCTURE ONLY.  Plain, slow, readable NumPy/SciPy code written from
the paper (arXiv:2504.01302) and from the standard definitions it cites.  It
shares no code with the CUDA path; only the seeded input generators in
``paper_2504_01302_b300.synth`` (which hold none of the method's arithmetic)
serve both.  Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it; the product path never does.

Every function cites the passage it follows.  Pins (tests/test_oracle_*.py)
tie it to closed forms, invariants, printed values and brute force.

Parity status per function is listed in the module headers; the ones with no
independent pin say "parity unpinned".
"""
