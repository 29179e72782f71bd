/*
 * CPU oracle for the longest-repeat (LR) query of Tian and Xu, "On Longest
 * Repeat Queries Using GPU" (arXiv 1501.06663).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path may call this code;
 * only the tests, the package's smoke check and the benchmark's CPU-baseline
 * leg do.  It shares no code, header or table with the CUDA library.
 *
 * Plain, slow and sequential on purpose: every function follows the paper's
 * definitions or algorithms step by step in the paper's notation, shifted to
 * 0-based indices:
 *   S[0..n), rank[i] = r iff sa[r] = i, lcp[0..n] with lcp[0] = lcp[n] = 0 and
 *   lcp[r] = |lcp(S[sa[r-1]..], S[sa[r]..])| (the paper's LCP[1..n+1], Sec. 3).
 * A repeat or LLR is reported as <start, length>; "does not exist" is
 * <-1, 0> (Algorithm 1).
 *
 * Readings taken where the paper is ambiguous:
 *  - all LR's of a position are listed by ascending start, so that the first
 *    one is the leftmost (Algorithm 3 prints them right to left, Algorithm 4
 *    left to right);
 *  - the rightward walk of Algorithms 2 and 4 stops at the first compact LLR
 *    that does not cover k, as its comment says; with strictly increasing
 *    starts and ends that is the first one whose start is past k (the printed
 *    test looks only at the end, which cannot fail on a rightward walk);
 *  - the compaction keeps LLR_i iff L_i > 0 and L_i >= L_{i-1} (Algorithm 2's
 *    one-pass rule and kernel K1 of Sec. 4.2.1), which drops exactly the
 *    L_i = L_{i-1} - 1 case of Sec. 3.2 by Lemma 2.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Lemma 1: L_i = max(LCP[Rank[i]], LCP[Rank[i]+1]); LLR_i exists iff L_i > 0. */
static int32_t llr_len(const int32_t* rank, const int32_t* lcp, int64_t i) {
    int32_t a = lcp[rank[i]], b = lcp[rank[i] + 1];
    return a > b ? a : b;
}

/* The raw LLR array LLRr[i] = |LLR_i| (Sec. 3.1, first loop of Algorithm 1). */
void oracle_llr_raw(const int32_t* rank, const int32_t* lcp, int64_t n, int32_t* llrr) {
    for (int64_t i = 0; i < n; ++i) llrr[i] = llr_len(rank, lcp, i);
}

/*
 * Kernels K1 and K2 of Sec. 4.2.1 written sequentially: Flag[0] = 1 iff
 * LLRr[0] > 0; Flag[i] = 1 iff LLRr[i] > 0 and LLRr[i] >= LLRr[i-1];
 * Prefix_Sum[i] = Flag[0] + ... + Flag[i].  K3 then moves <i, LLRr[i]> to
 * LLRc[Prefix_Sum[i] - 1] (0-based) for every flagged i.  Returns the size of
 * LLRc.
 */
int64_t oracle_flag_prefix_scatter(const int32_t* llrr, int64_t n, int32_t* flag, int64_t* prefix,
                                   int32_t* c_start, int32_t* c_len) {
    int64_t run = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (i == 0) flag[i] = llrr[0] > 0;
        else flag[i] = llrr[i] > 0 && llrr[i] >= llrr[i - 1];
        run += flag[i];
        prefix[i] = run;
    }
    for (int64_t i = 0; i < n; ++i) {
        if (flag[i]) { c_start[prefix[i] - 1] = (int32_t)i; c_len[prefix[i] - 1] = llrr[i]; }
    }
    return run;
}

/* The one-pass compaction of Algorithms 2 and 4: keep <i, L> iff L > 0 and
 * L >= prev, where prev is the previous position's L.  Returns the size. */
int64_t oracle_compact(const int32_t* rank, const int32_t* lcp, int64_t n, int32_t* c_start, int32_t* c_len) {
    int64_t j = 0;
    int32_t prev = 0;
    for (int64_t i = 0; i < n; ++i) {
        int32_t L = llr_len(rank, lcp, i);
        if (L > 0 && L >= prev) { c_start[j] = (int32_t)i; c_len[j] = L; ++j; }
        prev = L;
    }
    return j;
}

/*
 * Algorithm 1: the leftmost LR of every k from the raw LLR array.  Walk from
 * i = k to the left; stop at the first LLR_i that does not cover k
 * (i + LLRr[i] - 1 < k); keep <i, LLRr[i]> whenever LLRr[i] >= the best
 * length so far, so ties end on the leftmost.
 */
void oracle_lr_leftmost_raw(const int32_t* rank, const int32_t* lcp, int64_t n,
                            int32_t* lr_start, int32_t* lr_len) {
    int32_t* llrr = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    oracle_llr_raw(rank, lcp, n, llrr);
    for (int64_t k = 0; k < n; ++k) {
        int32_t best_start = -1, best_len = 0;
        for (int64_t i = k; i >= 0; --i) {
            if (i + llrr[i] - 1 < k) break;
            else if (llrr[i] >= best_len) { best_start = (int32_t)i; best_len = llrr[i]; }
        }
        lr_start[k] = best_start; lr_len[k] = best_len;
    }
    free(llrr);
}

/*
 * Algorithm 3: all LR's of every k from the raw LLR array, two leftward walks
 * per k (the first finds the length, the second lists every LLR of that
 * length that covers k).  Output in CSR form: lr_len[k], lr_start[k] (the
 * leftmost, -1 if none), offsets[k..k+1) into starts (ascending start).
 * Writes at most `cap` starts; returns the total number, so a caller whose
 * buffer was too small can retry with a larger one.
 */
int64_t oracle_lr_all_raw(const int32_t* rank, const int32_t* lcp, int64_t n,
                          int32_t* lr_len, int32_t* lr_start, int64_t* offsets,
                          int32_t* starts, int64_t cap) {
    int32_t* llrr = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    oracle_llr_raw(rank, lcp, n, llrr);
    int64_t total = 0;
    offsets[0] = 0;
    for (int64_t k = 0; k < n; ++k) {
        int32_t length = 0;
        for (int64_t i = k; i >= 0; --i) {
            if (i + llrr[i] - 1 < k) break;
            else if (llrr[i] >= length) length = llrr[i];
        }
        int64_t first = total;
        if (length > 0) {
            for (int64_t i = k; i >= 0; --i) {
                if (i + llrr[i] - 1 < k) break;
                else if (llrr[i] == length) {
                    if (total < cap) starts[total] = (int32_t)i;
                    ++total;
                }
            }
            /* the walk met them right to left: list them left to right */
            int64_t hi = (total < cap ? total : cap) - 1;
            for (int64_t a = first; a < hi; ++a, --hi) {
                int32_t t = starts[a]; starts[a] = starts[hi]; starts[hi] = t;
            }
        }
        lr_len[k] = length;
        lr_start[k] = (length > 0 && first < cap) ? starts[first] : -1;
        offsets[k + 1] = total;
    }
    free(llrr);
    return total;
}

/*
 * Binary search of Algorithms 2 and 4: the smallest index t of LLRc whose
 * element covers k (start <= k <= start + length - 1), or -1.  Starts and
 * ends of LLRc strictly increase (Sec. 3.2), so the elements whose end is
 * >= k form a suffix, and the first of them covers k iff its start <= k.
 */
static int64_t first_cover(const int32_t* c_start, const int32_t* c_len, int64_t m, int64_t k) {
    int64_t lo = 0, hi = m;                 /* first t with end_t >= k */
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if ((int64_t)c_start[mid] + c_len[mid] - 1 >= k) hi = mid; else lo = mid + 1;
    }
    if (lo < m && c_start[lo] <= k) return lo;
    return -1;
}

/*
 * Algorithm 2: the leftmost LR of every k from the compact LLR array: binary
 * search for the first LLRc element covering k, then walk right while the
 * element covers k, taking a strictly longer one each time.
 */
void oracle_lr_leftmost_compact(const int32_t* rank, const int32_t* lcp, int64_t n,
                                int32_t* lr_start, int32_t* lr_len) {
    int32_t* cs = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    int32_t* cl = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    int64_t size = oracle_compact(rank, lcp, n, cs, cl);
    for (int64_t k = 0; k < n; ++k) {
        int32_t best_start = -1, best_len = 0;
        int64_t start = first_cover(cs, cl, size, k);
        if (start != -1) {
            for (int64_t i = start; i < size; ++i) {
                if (!(cs[i] <= k && (int64_t)cs[i] + cl[i] - 1 >= k)) break;
                else if (cl[i] > best_len) { best_start = cs[i]; best_len = cl[i]; }
            }
        }
        lr_start[k] = best_start; lr_len[k] = best_len;
    }
    free(cs); free(cl);
}

/*
 * Algorithm 4: all LR's of every k from the compact LLR array (binary search,
 * then two rightward walks).  Same CSR output and return value as
 * oracle_lr_all_raw; the walk already meets the LR's left to right.
 */
int64_t oracle_lr_all_compact(const int32_t* rank, const int32_t* lcp, int64_t n,
                              int32_t* lr_len, int32_t* lr_start, int64_t* offsets,
                              int32_t* starts, int64_t cap) {
    int32_t* cs = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    int32_t* cl = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    int64_t size = oracle_compact(rank, lcp, n, cs, cl);
    int64_t total = 0;
    offsets[0] = 0;
    for (int64_t k = 0; k < n; ++k) {
        int32_t length = 0;
        int64_t first = total;
        int64_t start = first_cover(cs, cl, size, k);
        if (start != -1) {
            for (int64_t i = start; i < size; ++i) {
                if (!(cs[i] <= k && (int64_t)cs[i] + cl[i] - 1 >= k)) break;
                else if (cl[i] > length) length = cl[i];
            }
            for (int64_t i = start; i < size; ++i) {
                if (!(cs[i] <= k && (int64_t)cs[i] + cl[i] - 1 >= k)) break;
                else if (cl[i] == length) {
                    if (total < cap) starts[total] = cs[i];
                    ++total;
                }
            }
        }
        lr_len[k] = length;
        lr_start[k] = (length > 0 && first < cap) ? starts[first] : -1;
        offsets[k + 1] = total;
    }
    free(cs); free(cl);
    return total;
}

/*
 * Walk statistics of Table 2, per position k:
 *   alpha[k] = the raw LLR's that Algorithm 1's leftward walk from k meets
 *              and that cover k (the walk stops at the first that does not);
 *   beta[k]  = the compact LLR's that Algorithm 2's rightward walk from the
 *              binary-search result meets and that cover k.
 * Lemma 1 of the paper and the statement of Algorithm 2 call their averages
 * alpha and beta: the number of LLR's (raw, compact) covering a position.
 * Returns the size of LLRc.
 */
int64_t oracle_walk_counts(const int32_t* rank, const int32_t* lcp, int64_t n, int32_t* alpha, int32_t* beta) {
    int32_t* llrr = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    int32_t* cs = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    int32_t* cl = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    oracle_llr_raw(rank, lcp, n, llrr);
    int64_t size = oracle_compact(rank, lcp, n, cs, cl);
    for (int64_t k = 0; k < n; ++k) {
        int32_t a = 0;
        for (int64_t i = k; i >= 0; --i) {
            if (i + llrr[i] - 1 < k) break;
            ++a;
        }
        int32_t b = 0;
        int64_t start = first_cover(cs, cl, size, k);
        if (start != -1) {
            for (int64_t i = start; i < size; ++i) {
                if (!(cs[i] <= k && (int64_t)cs[i] + cl[i] - 1 >= k)) break;
                ++b;
            }
        }
        alpha[k] = a;
        beta[k] = b;
    }
    free(llrr); free(cs); free(cl);
    return size;
}

/*
 * Algorithm 3 for a sample of positions only (for spot checks on strings too
 * long to run in full): for each ks[q], the two leftward walks over the raw
 * LLR array, with LLRr[i] computed on demand by Lemma 1.  Returns the total
 * number of LR starts; they are written ascending, per sample, into `starts`
 * (at most cap), with offsets[q..q+1) delimiting sample q.
 */
int64_t oracle_lr_at(const int32_t* rank, const int32_t* lcp, int64_t n, const int64_t* ks, int64_t nk,
                     int32_t* lr_len, int32_t* lr_start, int64_t* offsets, int32_t* starts, int64_t cap) {
    int64_t total = 0;
    offsets[0] = 0;
    for (int64_t q = 0; q < nk; ++q) {
        int64_t k = ks[q];
        int32_t length = 0;
        for (int64_t i = k; i >= 0; --i) {
            int32_t L = llr_len(rank, lcp, i);
            if (i + L - 1 < k) break;
            else if (L >= length) length = L;
        }
        int64_t first = total;
        if (length > 0) {
            for (int64_t i = k; i >= 0; --i) {
                int32_t L = llr_len(rank, lcp, i);
                if (i + L - 1 < k) break;
                else if (L == length) {
                    if (total < cap) starts[total] = (int32_t)i;
                    ++total;
                }
            }
            int64_t hi = (total < cap ? total : cap) - 1;
            for (int64_t a = first; a < hi; ++a, --hi) {
                int32_t t = starts[a]; starts[a] = starts[hi]; starts[hi] = t;
            }
        }
        lr_len[q] = length;
        lr_start[q] = (length > 0 && first < cap) ? starts[first] : -1;
        offsets[q + 1] = total;
    }
    return total;
}

/*
 * The problem statement itself, from the string alone (Sec. 2, Definition 1):
 * no suffix array, no lemma.  A substring S[i..i+l-1] is a repeat iff some
 * other start i' != i has an equal substring, i.e. iff l <= maxrep[i], the
 * longest common prefix of suffix i with any other suffix.  maxrep comes
 * from comparing every pair of suffixes along each diagonal i' - i = d,
 * right to left: lcp(i, i+d) = S[i] == S[i+d] ? 1 + lcp(i+1, i+1+d) : 0.
 * Every prefix of a repeat is a repeat, so the longest repeat starting at i
 * that covers k is S[i..i+maxrep[i]-1] when i <= k <= i + maxrep[i] - 1, and
 * LR_k is the longest of those; all LR's of k are all such i of that length.
 * O(n^2) time; for short strings only.  Same CSR output as the walks.
 */
int64_t oracle_brute(const uint8_t* s, int64_t n, int32_t* lr_len, int32_t* lr_start,
                     int64_t* offsets, int32_t* starts, int64_t cap) {
    int32_t* maxrep = (int32_t*)calloc((size_t)(n ? n : 1), sizeof(int32_t));
    for (int64_t d = 1; d < n; ++d) {
        int32_t run = 0;
        for (int64_t i = n - 1 - d; i >= 0; --i) {
            run = (s[i] == s[i + d]) ? run + 1 : 0;      /* lcp of suffixes i and i+d */
            if (run > maxrep[i]) maxrep[i] = run;
            if (run > maxrep[i + d]) maxrep[i + d] = run;
        }
    }
    int64_t total = 0;
    offsets[0] = 0;
    for (int64_t k = 0; k < n; ++k) {
        int32_t length = 0;
        for (int64_t i = 0; i <= k; ++i)
            if (maxrep[i] > 0 && i + maxrep[i] - 1 >= k && maxrep[i] > length) length = maxrep[i];
        int64_t first = total;
        if (length > 0)
            for (int64_t i = 0; i <= k; ++i)
                if (maxrep[i] == length && i + maxrep[i] - 1 >= k) {
                    if (total < cap) starts[total] = (int32_t)i;
                    ++total;
                }
        lr_len[k] = length;
        lr_start[k] = (length > 0 && first < cap) ? starts[first] : -1;
        offsets[k + 1] = total;
    }
    free(maxrep);
    return total;
}
