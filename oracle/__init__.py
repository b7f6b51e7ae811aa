"""CPU oracle for REWL on the 2D Potts model -- test infrastructure only.

Only the tests, the package smoke check and the benchmark's CPU-baseline leg
may import this package.  The product library never does.
"""
