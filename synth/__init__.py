"""Seeded synthetic inputs shared by the oracle tests, the CUDA path's tests and the benchmark.

This package holds none of the method's arithmetic (no system matrix, no block
operators, no sampling, no solver).  It simulates a scanner: random ellipse /
ellipsoid phantoms, their exact line integrals along each measurement line
(its own ray generator, written independently of the oracle and of the
library), pixel averages of the phantom for error measures, measurement noise,
and the workload definitions (geometry sizes, partitions, solver settings).

The paper does not print its phantom (the images of Sec. III are missing), so
every phantom here is a seeded stand-in with the sizes of the paper's runs.
"""
