"""GB300-native RNS-CKKS hot path of HEAR / Fast-HEAR (arXiv 2104.09164)."""
