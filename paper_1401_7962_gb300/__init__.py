"""GB300-native Gauss-Jordan inversion (arXiv:1401.7962) -- Python binding of the C-ABI library."""
