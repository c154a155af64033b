"""FP64 CPU oracle for the CSGD / GCSGD block solver (Gao & Blumensath, Sec. II).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import, call,
link or execute anything in this package.  The product path (the CUDA library
``paper_1709_00953_gb300``) never touches it, and this package never touches the
product: the two share no code, headers, tables or helpers.  The seeded input
generators in ``synth`` are the only thing both sides use.

Modules, each following the paper's definitions in plain FP64:

``geometry``  scan geometries and the rays of every measurement (Sec. II-D, Sec. III)
``siddon``    A_i^j = length of ray i inside voxel j, by the alpha-merge (Sec. II-A)
``blocks``    row blocks I, column blocks J and the operators A_I^J, (A_I^J)^T (Eq. e1)
``ptable``    the importance table P(I,J) = P_S / P_T (Sec. II-C, Alg. 3)
``schedule``  the random choice of (I, J) blocks and groups (Alg. 3, Alg. 4, Sec. III-D)
``solver``    Alg. 1 (basic iteration) inside Alg. 2 / 3 / 4
``metrics``   SNR, observation gap, RMSE (Sec. III)

Parity status of each function is stated in its docstring; the pins live in
``tests/test_oracle_*.py``.
"""
