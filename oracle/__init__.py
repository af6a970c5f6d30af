"""CPU oracle for IFEAST: test infrastructure, not part of the product.

Only the test suite, the smoke check and the CPU-baseline legs of the bench
script may import this package. Nothing in ``paper_1706_00692_gb300`` imports
it, and it imports nothing from there.
"""
