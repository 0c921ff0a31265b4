/* Uniform ORB features on the GPU: detection, description and template-to-live matching.
 *
 * Section 2.1 (first paragraph) of Zhou & Jagadeesan, "Real-time Surface Deformation Recovery
 * from Stereo Videos": FAST corners are detected on the GPU and a corner is suppressed when a
 * neighbouring pixel has a larger corner response, which spreads the features over low-texture
 * areas; every live frame is then matched against the template's features, which gives the
 * two 3D point sets o1 (template) and o2 (live) of Eq. 2. The matches feed ds_submit_frame
 * (defsolve.h) directly.
 *
 * The method's details, where the paper leaves them open:
 *   - 8-bit grey-level images, row-major H x W;
 *   - FAST-9: the 16 pixels of the radius-3 digital circle; a pixel p is a corner iff 9
 *     cyclically contiguous circle pixels are all brighter than I_p + fast_t or all darker than
 *     I_p - fast_t; response V = max(sum over brighter pixels of (I_c - I_p - fast_t), sum over
 *     darker pixels of (I_p - I_c - fast_t));
 *   - suppression: a corner is dropped iff one of its 8 neighbours has a strictly larger
 *     response (equal responses both stay); keypoints lie at least `border` pixels from every
 *     edge and, when a depth map is given, on pixels of positive depth; they are listed in
 *     ascending pixel index, the first max_kp kept;
 *   - orientation: intensity centroid over the disc of radius 15, theta = atan2(m01, m10) in
 *     FP64, bin = rint(theta / (2 pi / 32)) mod 32;
 *   - descriptor: 256 binary tests on 5 x 5 box sums S; test i uses the pattern's pair i
 *     (a_i, b_i), rotated by 2 pi bin / 32 and rounded to integer offsets (FP64, ties to even):
 *     bit i = S(p + a_i) < S(p + b_i), stored as bit i % 32 of 32-bit word i / 32;
 *   - matching: Hamming distance; template keypoint t and live keypoint l match iff each is the
 *     other's nearest (ties to the lower index) and the distance is <= max_dist; matches are
 *     listed in ascending t; o2 = the live keypoint back-projected by the live depth,
 *     ((u - cx) z / fx, (v - cy) z / fy, z).
 *
 * Memory: every ds_orb owns its device buffers (image, depth, response and box-sum maps,
 * keypoints, descriptors, matches); inputs may be host or device pointers and are copied in
 * before the call returns its status. Calls are asynchronous on the object's stream unless they
 * return counts or copy results to the host. Status codes are those of defsolve.h.
 */
#ifndef DEFSOLVE_ORB_H
#define DEFSOLVE_ORB_H

#include <stdint.h>

#include "defsolve.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t fast_t;    /* FAST threshold on grey levels, 0..255 (default 20)                      */
  int32_t border;    /* keypoints at least this many pixels from every edge, >= 16 (default 16)
                      * (the orientation disc and the rotated tests with their box sums fit)    */
  int32_t max_dist;  /* largest Hamming distance of a match, 0..256 (default 64)                 */
  int32_t max_kp;    /* keypoints kept per image, 1..W*H (0 = default W * H / 8)                 */
} ds_orb_params;

typedef struct ds_orb_s* ds_orb;

/* Fills *p with the defaults above. */
void ds_orb_default_params(ds_orb_params* p);

/* Creates a feature context for W x H images (W, H in [40, 4096]) seen through K (used to
 * back-project live keypoints). pattern: 256 x 4 doubles (ax, ay, bx, by per test), every point
 * within 13 pixels of the origin; copied. p may be NULL (defaults). cuda_stream: a cudaStream_t
 * or NULL for a stream owned by the context.
 * Errors: DS_ERR_ARG (sizes, parameters, a pattern point out of range), DS_ERR_OOM, DS_ERR_CUDA. */
int ds_orb_create(int32_t W, int32_t H, ds_intrinsics K, const ds_orb_params* p,
                  const double* pattern, void* cuda_stream, ds_orb* out);

/* Detects and describes the keypoints of one image (H x W bytes). depth_hw (H x W floats, may be
 * NULL): when given, keypoints need positive depth there, and the depth is kept for matching
 * (this context as the live side). Asynchronous. Errors: DS_ERR_ARG, DS_ERR_CUDA. */
int ds_orb_detect(ds_orb o, const uint8_t* image_hw, const float* depth_hw);

/* Synchronises; *n_kept = keypoints stored (<= max_kp), *n_total = keypoints found. Either
 * pointer may be NULL. */
int ds_orb_num_keypoints(ds_orb o, int32_t* n_kept, int32_t* n_total);

/* Copies the stored keypoints to host arrays of n_kept entries: pixel index, response,
 * orientation bin, and 8 descriptor words each. Any pointer may be NULL. Synchronises. */
int ds_orb_get_keypoints(ds_orb o, int32_t* pix, int32_t* score, int32_t* bin, uint32_t* desc_8);

/* Matches the keypoints of `tmpl` (detected once on the template image) to those of `live`
 * (detected with its depth), on live's stream after tmpl's pending work; tmpl's stream then waits
 * for the match, so a later ds_orb_detect on tmpl cannot overwrite what it reads. The results
 * stay in `live`. Both contexts must have the same pattern; tmpl and live may be the same
 * object.
 * Errors: DS_ERR_ARG (NULL, different image sizes), DS_ERR_STATE (nothing detected, or no live
 * depth), DS_ERR_CUDA. */
int ds_orb_match(ds_orb tmpl, ds_orb live);

/* Synchronises; *M = number of matches of the last ds_orb_match on `live`. */
int ds_orb_num_matches(ds_orb live, int32_t* M);

/* Copies the M matches to host arrays: template keypoint index, live keypoint index, Hamming
 * distance, template pixel (o1's pixel) and the live 3D point (3 floats, o2). Any pointer may be
 * NULL. Synchronises. */
int ds_orb_get_matches(ds_orb live, int32_t* tmpl_kp, int32_t* live_kp, int32_t* dist,
                       int32_t* tmpl_pixel, float* xyz_3);

/* Device pointers of the match arrays (template pixel per match, M x 3 live points), valid
 * until the next ds_orb_match or ds_orb_destroy on `live`: pass them with M to ds_submit_frame
 * (which reads device pointers in place, on its own stream: synchronise first, e.g. with
 * ds_orb_num_matches). */
int ds_orb_match_device(ds_orb live, const int32_t** tmpl_pixel, const float** xyz_3);

int ds_orb_destroy(ds_orb o);

#ifdef __cplusplus
}
#endif

#endif /* DEFSOLVE_ORB_H */
