"""FP64 CPU oracle of the hybrid LB-FD coupled step (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The product path (``paper_2311_15242_gb300``)
never imports it and shares no code with it.
"""
