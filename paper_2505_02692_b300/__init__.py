"""B300-native engine for the fastabx ABX distance and score path.

Importing the package is cheap; the CUDA library is loaded on first use by
``paper_2505_02692_b300.abx``.
"""
